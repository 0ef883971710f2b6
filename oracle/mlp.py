"""Slice-level selector network (oracle; test infrastructure only).

The paper picks the number of slices by hand or with the library's automatic mode, and reports
accuracy against the slice count (sections "Theory of emulated FP64 arithmetic" and "Numerical
procedure", the eager and performant modes).  The learned selector of this project predicts, for
one emulated product, log10 of its relative error at every slice level from statistics of its
operands' exponents.  This module is the plain definition of that network and its training step:

    H1 = tanh(X W1 + b1),  H2 = tanh(H1 W2 + b2),  Y = H2 W3 + b3,
    loss = sum(M * (Y - T)^2) / max(1, sum(M))        (M masks missing targets)

with the gradients written out by the chain rule, and one Adam step (Kingma and Ba, 2015:
m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)).
Parameters are flattened as W1 (row-major nin x nh), b1, W2, b2, W3, b3.

Parity: pinned (tests/test_oracle_mlp.py) by central finite differences of the loss.
"""
from __future__ import annotations

import numpy as np


def shapes(nin: int, nh: int, nout: int):
    return [(nin, nh), (nh,), (nh, nh), (nh,), (nh, nout), (nout,)]


def unflatten(flat, nin: int, nh: int, nout: int):
    out, o = [], 0
    for sh in shapes(nin, nh, nout):
        k = int(np.prod(sh))
        out.append(np.asarray(flat[o:o + k]).reshape(sh))
        o += k
    return out


def flatten(parts):
    return np.concatenate([np.asarray(p).reshape(-1) for p in parts])


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = params
    H1 = np.tanh(X @ W1 + b1)
    H2 = np.tanh(H1 @ W2 + b2)
    return H2 @ W3 + b3, (H1, H2)


def loss_and_grads(params, X, T, M):
    """(loss, [dW1, db1, dW2, db2, dW3, db3])."""
    W1, b1, W2, b2, W3, b3 = params
    Y, (H1, H2) = forward(params, X)
    den = max(1.0, float(M.sum()))
    R = M * (Y - T)
    loss = float((R * (Y - T)).sum() / den)
    dY = 2.0 * R / den
    dW3 = H2.T @ dY
    db3 = dY.sum(axis=0)
    dZ2 = (dY @ W3.T) * (1.0 - H2 * H2)
    dW2 = H1.T @ dZ2
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2.T) * (1.0 - H1 * H1)
    dW1 = X.T @ dZ1
    db1 = dZ1.sum(axis=0)
    return loss, [dW1, db1, dW2, db2, dW3, db3]


def adam_step(flat, grad, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update of the flat parameter vector (returns new flat, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
