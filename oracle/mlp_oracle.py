"""FP64 reference of the candidate-budget network -- TEST INFRASTRUCTURE ONLY.

The paper trains a model offline to choose its cache split (Section 5.2,
"we train a model"); it prints no network.  The library's learned part is a
small multilayer perceptron that predicts, from a query's features, the level
at which the collision-counting loop will stop.  This module is the plain
numpy FP64 definition of that network, its loss and its gradients, used only
by the tests to check the library's CUDA forward and backward kernels.  It
shares no code with the library.

Network: x (n_in) -> ReLU(W1 x + b1) (H) -> ReLU(W2 h1 + b2) (H) -> W3 h2 + b3
(C logits); loss = mean over the batch of -log softmax(logits)[y].
Flat parameter layout (the library's): W1 (H x n_in, row-major), b1 (H),
W2 (H x H), b2 (H), W3 (C x H), b3 (C).
"""
from __future__ import annotations

import numpy as np


def param_count(n_in: int, hidden: int, classes: int) -> int:
    return hidden * n_in + hidden + hidden * hidden + hidden + classes * hidden + classes


def unpack(p: np.ndarray, n_in: int, hidden: int, classes: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = []
    for shape in ((hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (classes, hidden),
                  (classes,)):
        size = int(np.prod(shape))
        out.append(p[o:o + size].reshape(shape))
        o += size
    return out


def loss_and_grad(p: np.ndarray, X: np.ndarray, y: np.ndarray, n_in: int, hidden: int,
                  classes: int):
    """Mean cross-entropy and its gradient (flat, library layout), FP64."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, hidden, classes)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    z3 = a2 @ W3.T + b3
    zmax = z3.max(axis=1, keepdims=True)
    e = np.exp(z3 - zmax)
    s = e.sum(axis=1, keepdims=True)
    logp = (z3 - zmax) - np.log(s)
    loss = -float(np.mean(logp[np.arange(n), y]))
    prob = e / s
    d3 = prob.copy()
    d3[np.arange(n), y] -= 1.0
    d3 /= n
    gW3 = d3.T @ a2
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3) * (z2 > 0)
    gW2 = d2.T @ a1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, grad


def predict_proba(p: np.ndarray, X: np.ndarray, n_in: int, hidden: int, classes: int):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, hidden, classes)
    a1 = np.maximum(np.asarray(X, np.float64) @ W1.T + b1, 0.0)
    a2 = np.maximum(a1 @ W2.T + b2, 0.0)
    z3 = a2 @ W3.T + b3
    e = np.exp(z3 - z3.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)
