"""Training data and training of the slice-level selector network (argument marshalling over the
C ABI: the products, errors, features and the network's forward/backward/Adam all run in the
library's kernels)."""
from __future__ import annotations

import numpy as np
import torch

from . import Heff, MLP

LEVELS = tuple(range(3, 9))   # levels the network predicts (log10 relative error at each)
ERR_FLOOR = 1e-19             # errors below this (exact at the reference level) are clamped


def harvest(h: Heff, psi: torch.Tensor, levels=LEVELS):
    """(X, T, M) rows for every product of ``h``: features, log10 relative error at every level
    (measured on the device against the handle's own level), mask.  The handle should be built
    with slices = 9 and level = 8 so that the reference is 8 slices deep."""
    f1, f2 = h.problem_features(psi)
    errs = [h.problem_errors(psi, lev) for lev in levels]
    X, T, M = [], [], []
    for stage, f in ((0, f1), (1, f2)):
        for q in range(f.shape[0]):
            e = [errs[i][stage][q] for i in range(len(levels))]
            if e[0] < 0:          # no product for this sector
                continue
            X.append(f[q])
            T.append([np.log10(max(x, ERR_FLOOR)) for x in e])
            M.append([1.0] * len(levels))
    return (np.asarray(X, dtype=np.float32).reshape(-1, f1.shape[1]),
            np.asarray(T, dtype=np.float32).reshape(-1, len(levels)),
            np.asarray(M, dtype=np.float32).reshape(-1, len(levels)))


def train(X, T, M, epochs=400, batch=64, lr=2e-3, seed=4, nhidden=64, device="cuda") -> MLP:
    """A selector network trained on the device (Adam, shuffled minibatches)."""
    net = MLP(nin=X.shape[1], nhidden=nhidden, nout=T.shape[1], seed=seed)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)
    net.train(d(X), d(T), d(M), epochs=epochs, batch=batch, lr=lr, seed=seed + 1)
    return net
