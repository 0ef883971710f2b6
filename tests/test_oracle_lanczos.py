"""Pins of the Lanczos oracle against numpy.linalg.eigh (with and without restarts)."""
import numpy as np

from oracle import lanczos


def test_lanczos_matches_eigh():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(150, 150))
    A = A + A.T
    lam, U = np.linalg.eigh(A)
    for krylov in (40, 12):                          # no restart needed / several restarts
        th, x, it, ok = lanczos.lanczos(lambda v: A @ v, rng.normal(size=150), eps=1e-10, max_iter=2000,
                                        krylov=krylov)
        assert ok
        assert abs(th - lam[0]) < 1e-9
        assert abs(abs(x @ U[:, 0]) - 1.0) < 1e-9
        assert np.linalg.norm(A @ x - th * x) < 1e-8


def test_lanczos_estimate_is_the_residual():
    rng = np.random.default_rng(1)
    A = np.diag(np.arange(60.0)) + 0.1 * rng.normal(size=(60, 60))
    A = A + A.T
    hist = []
    th, x, it, ok = lanczos.lanczos(lambda v: A @ v, np.ones(60), eps=1e-6, max_iter=300, krylov=60, history=hist)
    assert ok and hist[-1][1] <= 1e-6
    # without restarts the estimate beta_j |y_j| equals |A x - theta x|
    assert abs(np.linalg.norm(A @ x - th * x) - hist[-1][1]) < 1e-9
