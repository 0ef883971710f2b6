"""The MPO of the ab initio Hamiltonian (host code of the library) against the brute-force
Jordan-Wigner Fock-space Hamiltonian of the oracle: contracted, they are the same matrix."""
import ctypes as C

import numpy as np
import pytest

import synthetic
from oracle import fci


@pytest.fixture(scope="module")
def lib():
    from paper_2510_04795_gb300 import _native
    return _native.load()


@pytest.mark.parametrize("L,seed", [(2, 3), (3, 3), (4, 5)])
def test_mpo_contracts_to_fock_hamiltonian(lib, L, seed):
    h, eri = synthetic.integrals(L, seed=seed)
    out = np.zeros((4 ** L, 4 ** L))
    assert lib.oz_mpo_dense(h.ctypes.data, eri.ctypes.data, L, out.ctypes.data) == 0
    Hb = fci.fock_hamiltonian_bruteforce(h, eri)
    assert np.abs(out - Hb).max() <= 1e-14 * np.abs(Hb).max() * 4 ** L


def test_mpo_bond_dimension_grows_quadratically(lib):
    dims = {}
    for L in (6, 8, 10):
        h, eri = synthetic.integrals(L, seed=0)
        chi = np.zeros(L + 1, dtype=np.int32)
        assert lib.oz_mpo_bond_dims(h.ctypes.data, eri.ctypes.data, L, chi.ctypes.data) == 0
        assert chi[0] == 1 and chi[-1] == 1
        dims[L] = int(chi.max())
    # complementary-operator states: O(L^2) at the middle bond, far below the O(L^4) term count
    assert dims[10] < 2 * L ** 2 * 2 + 64
    assert dims[8] / dims[6] < (8 / 6) ** 2 * 1.5


def test_mpo_rejects_bad_sizes(lib):
    h = np.zeros((1, 1))
    eri = np.zeros(1)
    out = np.zeros(1)
    assert lib.oz_mpo_dense(h.ctypes.data, eri.ctypes.data, 5, out.ctypes.data) == 1
    chi = np.zeros(2, dtype=np.int32)
    assert lib.oz_mpo_bond_dims(h.ctypes.data, eri.ctypes.data, 1, chi.ctypes.data) == 1
