"""Pins of the FCI, Davidson and block-sparse H_eff oracles."""
import math

import numpy as np
import pytest
import torch

import synthetic
from oracle import davidson, fci, heff, ozaki


def test_fci_dimension_c0():
    # L = 8 orbitals, N = 8 electrons, Sz = 0: C(8,4)^2 = 4900 determinants
    assert len(fci.strings(8, 4)) ** 2 == 4900 == math.comb(8, 4) ** 2


def test_fci_noninteracting_closed_form():
    h, _ = synthetic.integrals(6, seed=11)
    eri = np.zeros((6,) * 4)
    E, _, H = fci.ground_state(h, eri, 6, 0)
    w = np.linalg.eigvalsh(h)
    assert abs(E - 2 * w[:3].sum()) < 1e-12


def test_fci_hubbard_dimer():
    for t, U in ((1.0, 4.0), (0.7, 1.3), (1.0, 0.0)):
        h = np.array([[0.0, -t], [-t, 0.0]])
        eri = np.zeros((2,) * 4)
        eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
        E, _, _ = fci.ground_state(h, eri, 2, 0)
        assert abs(E - (U / 2 - math.sqrt(U * U / 4 + 4 * t * t))) < 1e-12


@pytest.mark.parametrize("L,N,twosz", [(3, 2, 0), (3, 3, 1), (4, 4, 0), (4, 3, -1)])
def test_fci_vs_bruteforce_fock(L, N, twosz):
    h, eri = synthetic.integrals(L, seed=5 + L)
    E, _, _ = fci.ground_state(h, eri, N, twosz)
    Hf = fci.fock_hamiltonian_bruteforce(h, eri)
    assert np.allclose(Hf, Hf.T, atol=1e-12)
    idx = fci.sector_mask(L, N, twosz)
    Eb = np.linalg.eigvalsh(Hf[np.ix_(idx, idx)])[0]
    assert abs(E - Eb) < 1e-11


def test_davidson_random_symmetric():
    rng = np.random.default_rng(0)
    n = 300
    A = rng.normal(size=(n, n))
    A = 0.5 * (A + A.T) + np.diag(np.arange(n) * 0.5)
    theta, x, it, ok = davidson.davidson(lambda v: A @ v, np.diag(A), rng.normal(size=n), tol=1e-10)
    assert ok
    w, V = np.linalg.eigh(A)
    assert abs(theta - w[0]) < 1e-10
    assert abs(abs(x @ V[:, 0]) - 1) < 1e-10


def _tiny_problem(spread=True, seed=1, grid=(3, 3), dims=(2, 6), nterms=8):
    st = synthetic.heff_structure(grid=grid, dims=dims, nterms=nterms, spread=spread, seed=seed)
    Lb, Rb = zip(*[synthetic.gen_task_blocks(st, t) for t in range(st.ntask)])
    Lb = [x.numpy() for x in Lb]
    Rb = [x.numpy() for x in Rb]
    psi = synthetic.gen_psi(st).numpy()
    return st, Lb, Rb, psi


def test_heff_blocks_match_kronecker_bruteforce():
    st, Lb, Rb, psi = _tiny_problem()
    H = heff.heff_dense(st, Lb, Rb)
    y = heff.heff_apply_fp64(st, Lb, Rb, psi)
    assert np.allclose(y, H @ psi, rtol=0, atol=1e-13 * np.abs(H).sum())


def test_heff_symmetric():
    st, Lb, Rb, psi = _tiny_problem(seed=3)
    H = heff.heff_dense(st, Lb, Rb)
    assert np.allclose(H, H.T, rtol=0, atol=1e-14 * np.abs(H).max())
    rng = np.random.default_rng(0)
    x, y = rng.normal(size=psi.size), rng.normal(size=psi.size)
    hx, hy = heff.heff_apply_fp64(st, Lb, Rb, x), heff.heff_apply_fp64(st, Lb, Rb, y)
    assert abs(x @ hy - hx @ y) <= 1e-13 * np.linalg.norm(hx) * np.linalg.norm(y)


def test_heff_diag_is_diagonal_of_dense():
    # the Davidson preconditioner: diagonal of the brute-force Kronecker sum (no other task touches it)
    st, Lb, Rb, psi = _tiny_problem(seed=6)
    H = heff.heff_dense(st, Lb, Rb)
    d = heff.heff_diag(st, Lb, Rb)
    assert np.allclose(d, np.diag(H), rtol=1e-15, atol=1e-15 * np.abs(H).max())
    assert np.count_nonzero(d) > 0


def test_davidson_history_and_restart():
    # a small subspace forces restarts; the answer still matches eigh and the residuals reach tol
    st, Lb, Rb, psi = _tiny_problem(spread=False, seed=4, grid=(3, 2), dims=(3, 8))
    H = heff.heff_dense(st, Lb, Rb)
    hist = []
    theta, x, it, ok = davidson.davidson(lambda v: H @ v, np.diag(H), psi, tol=1e-9, max_sub=8, history=hist)
    assert ok and it > 8 and len(hist) == it and hist[-1][1] <= 1e-9
    assert abs(theta - np.linalg.eigvalsh(H)[0]) < 1e-9
    # Ritz values of a growing or restarted Krylov-like subspace never rise (Cauchy interlacing)
    th = [h[0] for h in hist]
    assert all(b <= a + 1e-12 for a, b in zip(th, th[1:]))


def test_davidson_on_dense_heff():
    st, Lb, Rb, psi = _tiny_problem(spread=False, seed=4, grid=(3, 2), dims=(3, 8))
    H = heff.heff_dense(st, Lb, Rb)
    theta, x, it, ok = davidson.davidson(lambda v: heff.heff_apply_fp64(st, Lb, Rb, v), np.diag(H), psi,
                                         tol=1e-10, max_sub=12)
    assert ok
    assert abs(theta - np.linalg.eigvalsh(H)[0]) < 1e-10


def test_heff_emulated_close_to_fp64():
    st, Lb, Rb, psi = _tiny_problem(seed=5)
    yref = heff.heff_apply_fp64(st, Lb, Rb, psi)
    errs = [heff.rel_frobenius(heff.heff_apply_emulated(st, Lb, Rb, psi, 7, s), yref) for s in (3, 4, 5, 7)]
    assert errs[-1] < 1e-13
    assert errs[0] > errs[1] > errs[2] > errs[3]


def test_heff_emulated_invariant_to_task_order():
    st, Lb, Rb, psi = _tiny_problem(seed=6)
    y1 = heff.heff_apply_emulated(st, Lb, Rb, psi, 4)
    perm = np.random.default_rng(0).permutation(st.ntask)
    st2 = synthetic.HeffStructure(st.labels, st.m, st.n, st.term_delta, st.term_coef, st.tasks[perm],
                                  st.spread, st.seed)
    y2 = heff.heff_apply_emulated(st2, [Lb[i] for i in perm], [Rb[i] for i in perm], psi, 4)
    assert np.array_equal(y1, y2)


@pytest.mark.parametrize("S", [3, 7])
def test_heff_entries_match_whole_emulated_product(S):
    # single entries from the operand rows they depend on equal the whole two-stage definition,
    # entry by entry (spread exponents, so a wrong row or column exponent would show)
    st, Lb, Rb, psi = _tiny_problem(seed=7)
    y = heff.heff_apply_emulated(st, Lb, Rb, psi, S)
    off = st.psi_offsets()
    P = {q: psi[off[q]:off[q + 1]].reshape(int(st.m[q]), int(st.n[q])) for q in range(st.nsec)}
    checked = 0
    for q in range(st.nsec):
        into = [t for t in range(st.ntask) if int(st.tasks[t][2]) == q]
        m, n = int(st.m[q]), int(st.n[q])
        js = list(range(n))
        for i in range(m):
            L_rows = {t: Lb[t][i] for t in into}
            R_rows = {t: Rb[t][js] for t in into}
            got = heff.heff_entries_emulated(st, q, i, js, L_rows, R_rows, P, S)
            assert np.array_equal(got, y[off[q] + i * n: off[q] + (i + 1) * n])
            checked += n
    assert checked == psi.size


def test_synthetic_bit_reproducible_blocks():
    st = synthetic.heff_structure(grid=(3, 3), dims=(2, 6), nterms=8, seed=2)
    L0, R0 = synthetic.gen_task_blocks(st, 0)
    L1, R1 = synthetic.gen_task_blocks(st, 0)
    assert torch.equal(L0, L1) and torch.equal(R0, R1)
    # transpose partner
    p = int(st.partner[0])
    Lp, Rp = synthetic.gen_task_blocks(st, p)
    assert torch.equal(Lp, L0.T) and torch.equal(Rp, R0.T)
