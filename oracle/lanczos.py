"""Lanczos eigensolver for the lowest eigenpair (oracle; test infrastructure only).

Most of the paper's runs use Lanczos for the two-site update and stop at a Krylov threshold
epsilon (sections "Theory of TNS/DMRG ..." and "Numerical procedure").  A plain statement of
the method with full reorthogonalisation and explicit restart:

  v_0 = x0 / |x0|
  repeat (restart):
    for j = 0, 1, ...:  w = H v_j;  alpha_j = v_j . w
                        w <- w - V (V^T w), twice (classical Gram-Schmidt against v_0..v_j)
                        beta_j = |w|;  T_{j,j} = alpha_j,  T_{j,j+1} = T_{j+1,j} = beta_j
                        (theta, y) = lowest eigenpair of T_{0..j}
                        stop when beta_j |y_j| <= eps (converged), or at max_iter products, or
                        beta_j < 1e-14; after `krylov` vectors restart from x = V y
                        v_{j+1} = w / beta_j
Parity: pinned (tests/test_oracle_lanczos.py) against numpy.linalg.eigh.
"""
from __future__ import annotations

import numpy as np


def lanczos(matvec, x0, eps=1e-10, max_iter=500, krylov=30, history=None):
    """Returns (theta, x, products, converged)."""
    v = np.asarray(x0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    total = 0
    theta = 0.0
    while True:
        V = [v]
        alpha, beta = [], []
        while True:
            w = np.asarray(matvec(V[-1]), dtype=np.float64)
            alpha.append(float(V[-1] @ w))
            Vm = np.array(V).T
            for _ in range(2):
                w = w - Vm @ (Vm.T @ w)
            b = float(np.linalg.norm(w))
            beta.append(b)
            k = len(alpha)
            T = np.diag(alpha) + np.diag(beta[:k - 1], 1) + np.diag(beta[:k - 1], -1)
            ev, EV = np.linalg.eigh(T)
            theta, y = float(ev[0]), EV[:, 0]
            total += 1
            est = b * abs(y[-1])
            if history is not None:
                history.append((theta, est))
            x = Vm @ y
            if est <= eps:
                return theta, x / np.linalg.norm(x), total, True
            if total >= max_iter or b < 1e-14:
                return theta, x / np.linalg.norm(x), total, False
            if k == krylov:
                v = x / np.linalg.norm(x)
                break
            V.append(w / b)
