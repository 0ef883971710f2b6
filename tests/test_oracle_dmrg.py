"""Pins of the explicit-basis DMRG oracle: the orbital-major Hamiltonian against the brute-force
Fock-space Hamiltonian, FCI without truncation, and the variational behaviour with truncation."""
import numpy as np
import pytest

import synthetic
from oracle import dmrg, fci


@pytest.mark.parametrize("L,N,twosz", [(3, 3, 1), (3, 2, 0), (3, 4, 0), (2, 2, 2)])
def test_orbital_major_hamiltonian_is_fock_bruteforce(L, N, twosz):
    h, eri = synthetic.integrals(L, seed=1)
    H, pats = dmrg.orbital_major_hamiltonian(h, eri, N, twosz)
    Hb = fci.fock_hamiltonian_bruteforce(h, eri)
    assert np.abs(H.toarray() - Hb[np.ix_(pats, pats)]).max() < 1e-13
    assert sorted(pats) == sorted(fci.sector_mask(L, N, twosz))


def test_dmrg_without_truncation_is_fci():
    # D above every block dimension: after the first half-sweep the two-site space at the last
    # bond is the whole sector, and from then on every bond is exact
    L, N = 6, 6
    h, eri = synthetic.integrals(L, seed=0)
    e0 = fci.ground_state(h, eri, N, 0)[0]
    d = dmrg.ExplicitDMRG(h, eri, N, 0, D=4096)
    E = np.array(d.sweep(2))
    nb = L - 1
    assert np.all(np.abs(E[nb - 1:] - e0) < 1e-10)
    assert np.all(E >= e0 - 1e-10)


def test_dmrg_truncated_is_variational_and_decreasing():
    L, N = 6, 6
    h, eri = synthetic.integrals(L, seed=0)
    e0 = fci.ground_state(h, eri, N, 0)[0]
    d = dmrg.ExplicitDMRG(h, eri, N, 0, D=8)
    E = np.array(d.sweep(3)).reshape(3, 2, L - 1)
    assert np.all(E >= e0 - 1e-10)
    ends = E[:, 1, -1]                          # energy at the end of every sweep
    assert np.all(np.diff(ends) <= 1e-10)
    assert ends[-1] - e0 < 1.0


def test_select_kept_never_splits_a_multiplet():
    assert dmrg.select_kept([0.5, 0.2, 0.2, 0.2, 0.1], 3) == 1
    assert dmrg.select_kept([0.5, 0.2, 0.2, 0.2, 0.1], 4) == 4
    assert dmrg.select_kept([0.5, 0.2, 0.1, 1e-15], 8) == 3       # below 1e-14 is dropped
    assert dmrg.select_kept([0.5, 0.25, 0.25 * (1 - 1e-12), 0.1], 2) == 1


@pytest.mark.slow
def test_dmrg_c0_d64_against_fci():
    # L = N = 8: the middle bond's two-site space is the whole 4900-dimensional sector (exact);
    # D = 64 cuts the other bonds, whose energies stay above FCI
    L, N = 8, 8
    h, eri = synthetic.integrals(L, seed=0)
    e0 = fci.ground_state(h, eri, N, 0)[0]
    d = dmrg.ExplicitDMRG(h, eri, N, 0, D=64)
    E = np.array(d.sweep(2)).reshape(2, 2, L - 1)
    assert np.all(E >= e0 - 1e-10)
    assert abs(E[1, 0, 3] - e0) < 1e-10
    assert 0 < E[1, 1, -1] - e0 < 1e-2


def test_dmrg_emulated_density_matrices_at_seven_slices_is_fp64():
    # seven slices carry 55 bits: the emulated rho differs from the FP64 one by about 2^-56 of its
    # norm, far below the keep threshold, so the truncations and energies are those of FP64;
    # two slices (15 bits) move the energies visibly but keep them above FCI
    L, N = 6, 6
    h, eri = synthetic.integrals(L, seed=0)
    e0 = fci.ground_state(h, eri, N, 0)[0]
    ref = np.array(dmrg.ExplicitDMRG(h, eri, N, 0, D=8).sweep(2))
    e7 = np.array(dmrg.ExplicitDMRG(h, eri, N, 0, D=8, rdm=(7, 7)).sweep(2))
    assert np.max(np.abs(e7 - ref)) < 1e-10
    e2 = np.array(dmrg.ExplicitDMRG(h, eri, N, 0, D=8, rdm=(2, 2)).sweep(2))
    assert np.all(e2 >= e0 - 1e-10)
    assert np.max(np.abs(e2 - ref)) > 1e-9
