"""Davidson eigensolver for the lowest eigenpair (oracle; test infrastructure only).

The DMRG update solves the H_eff eigenproblem with a Krylov method, Davidson
or Lanczos (section "Theory of TNS/DMRG ...", second subroutine), stopping at a
residual threshold epsilon (section "Numerical procedure").  This is a plain
statement of Davidson's method:

  V = [x0/|x0|], W = H V
  repeat:  G = V^T W (symmetrised);  (theta, y) = lowest eigenpair of G
           x = V y,  r = W y - theta x;  stop when |r|_2 <= tol
           delta = r / (theta - diag(H))   (|theta - diag| floored at 1e-12, sign kept)
           orthogonalise delta against V twice (classical Gram-Schmidt), normalise, append
           when V reaches max_sub vectors, restart from the Ritz vectors of the 2 lowest
           eigenvalues of G.

Parity: pinned (tests/test_oracle_fci_davidson_heff.py) against numpy.linalg.eigh on
random symmetric matrices and on dense H_eff.
"""
from __future__ import annotations

import numpy as np


def davidson(matvec, diag, x0, tol=1e-10, max_iter=200, max_sub=24, history=None):
    """Returns (theta, x, iterations, converged).  If ``history`` is a list, (theta, |r|) of every
    iteration is appended to it."""
    diag = np.asarray(diag, dtype=np.float64)
    x = np.asarray(x0, dtype=np.float64).copy()
    x /= np.linalg.norm(x)
    V = [x]
    W = [np.asarray(matvec(x), dtype=np.float64)]
    theta = float(x @ W[0])
    for it in range(1, max_iter + 1):
        Vm, Wm = np.array(V).T, np.array(W).T
        G = Vm.T @ Wm
        G = 0.5 * (G + G.T)
        w, Y = np.linalg.eigh(G)
        theta, y = float(w[0]), Y[:, 0]
        x = Vm @ y
        r = Wm @ y - theta * x
        rn = float(np.linalg.norm(r))
        if history is not None:
            history.append((theta, rn))
        if rn <= tol:
            return theta, x / np.linalg.norm(x), it, True
        den = theta - diag
        small = np.abs(den) < 1e-12
        den = np.where(small, np.where(den < 0, -1e-12, 1e-12), den)
        d = r / den
        if len(V) >= max_sub:
            keep = Vm @ Y[:, :2]
            kw = Wm @ Y[:, :2]
            V = [keep[:, 0], keep[:, 1]]
            W = [kw[:, 0], kw[:, 1]]
            Vm = np.array(V).T
        for _ in range(2):
            d = d - Vm @ (Vm.T @ d)
        nd = np.linalg.norm(d)
        if nd < 1e-14:
            return theta, x / np.linalg.norm(x), it, False
        d /= nd
        V.append(d)
        W.append(np.asarray(matvec(d), dtype=np.float64))
    return theta, x / np.linalg.norm(x), max_iter, False
