"""Full CI of the ab initio Hamiltonian (oracle; test infrastructure only).

The paper checks DMRG energies against exact diagonalisation where it is
affordable (section "Numerical benchmark": the FCI reference of F2) and uses
the variational principle (section "Theory of TNS/DMRG ...": energies approach
the exact ground state from above).  This module is that exact reference for
the small synthetic systems.

H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps),
E_pq = sum_sigma a^+_{p sigma} a_{q sigma}, chemist notation, no core energy.
Determinants are (alpha string, beta string) bit masks with all alpha
spin-orbitals ordered before the beta ones, so that E_pq acts on each string
separately with the Jordan-Wigner sign of that string alone.  (Any orbital
ordering gives the same spectrum.)

Parity: pinned (tests/test_oracle_fci.py) by the closed form with (pq|rs)=0,
the Hubbard dimer energy U/2 - sqrt(U^2/4 + 4t^2), the sector dimension, and a
brute-force Jordan-Wigner Fock-space Hamiltonian on L <= 4.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def strings(L: int, n: int) -> list:
    return [sum(1 << i for i in c) for c in itertools.combinations(range(L), n)]


def _excitation(str_list, L):
    """Sparse matrices e_pq on one spin string space: <s'| a+_p a_q |s>."""
    idx = {s: i for i, s in enumerate(str_list)}
    dim = len(str_list)
    mats = {}
    for p in range(L):
        for q in range(L):
            rows, cols, vals = [], [], []
            for j, s in enumerate(str_list):
                if not (s >> q) & 1:
                    continue
                sign = -1 if bin(s & ((1 << q) - 1)).count("1") % 2 else 1
                s1 = s & ~(1 << q)
                if (s1 >> p) & 1:
                    continue
                sign *= -1 if bin(s1 & ((1 << p) - 1)).count("1") % 2 else 1
                s2 = s1 | (1 << p)
                rows.append(idx[s2]); cols.append(j); vals.append(float(sign))
            mats[p, q] = sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim))
    return mats


def hamiltonian(h: np.ndarray, eri: np.ndarray, nalpha: int, nbeta: int) -> sp.csr_matrix:
    """Sparse FCI Hamiltonian in the (alpha string) x (beta string) basis."""
    L = h.shape[0]
    sa, sb = strings(L, nalpha), strings(L, nbeta)
    ea, eb = _excitation(sa, L), _excitation(sb, L)
    Ia, Ib = sp.identity(len(sa), format="csr"), sp.identity(len(sb), format="csr")
    E = {(p, q): (sp.kron(ea[p, q], Ib) + sp.kron(Ia, eb[p, q])).tocsr() for p in range(L) for q in range(L)}
    k = h - 0.5 * np.einsum("prrs->ps", eri)
    H = sp.csr_matrix((len(sa) * len(sb),) * 2)
    for p in range(L):
        for q in range(L):
            if k[p, q] != 0.0:
                H = H + k[p, q] * E[p, q]
    for p in range(L):
        for q in range(L):
            W = sp.csr_matrix(H.shape)
            for r in range(L):
                for s in range(L):
                    if eri[p, q, r, s] != 0.0:
                        W = W + eri[p, q, r, s] * E[r, s]
            if W.nnz:
                H = H + 0.5 * (E[p, q] @ W)
    return H.tocsr()


def ground_state(h, eri, nelec: int, twosz: int = 0):
    """Lowest eigenpair in the sector (N = nelec, 2Sz = twosz)."""
    na, nb = (nelec + twosz) // 2, (nelec - twosz) // 2
    H = hamiltonian(h, eri, na, nb)
    if H.shape[0] <= 2000:
        w, v = np.linalg.eigh(H.toarray())
        return float(w[0]), v[:, 0], H
    w, v = spla.eigsh(H, k=1, which="SA", tol=1e-14, maxiter=100000)
    return float(w[0]), v[:, 0], H


# ---------------------------------------------------------------------------------------------
# brute-force Jordan-Wigner Fock space (independent pin of the string construction)
# ---------------------------------------------------------------------------------------------

def fock_hamiltonian_bruteforce(h, eri):
    """Dense H on the full Fock space of 2L spin-orbitals (orbital-major, up before down),
    built by applying every second-quantised term to every occupation bit string."""
    L = h.shape[0]
    nso = 2 * L
    dim = 1 << nso

    def apply(ops, state):
        sign = 1
        for (dag, so) in reversed(ops):
            occ = (state >> so) & 1
            if dag == occ:
                return 0, None
            sign *= -1 if bin(state & ((1 << so) - 1)).count("1") % 2 else 1
            state ^= 1 << so
        return sign, state

    H = np.zeros((dim, dim))
    for st in range(dim):
        for p in range(L):
            for q in range(L):
                for sg in range(2):
                    if h[p, q] == 0.0:
                        continue
                    sgn, new = apply([(1, 2 * p + sg), (0, 2 * q + sg)], st)
                    if sgn:
                        H[new, st] += h[p, q] * sgn
        for p, q, r, s in itertools.product(range(L), repeat=4):
            v = eri[p, q, r, s]
            if v == 0.0:
                continue
            for sg, tg in itertools.product(range(2), repeat=2):
                sgn, new = apply([(1, 2 * p + sg), (1, 2 * r + tg), (0, 2 * s + tg), (0, 2 * q + sg)], st)
                if sgn:
                    H[new, st] += 0.5 * v * sgn
    return H


def sector_mask(L: int, nelec: int, twosz: int) -> np.ndarray:
    idx = []
    for st in range(1 << (2 * L)):
        na = sum((st >> (2 * p)) & 1 for p in range(L))
        nb = sum((st >> (2 * p + 1)) & 1 for p in range(L))
        if na + nb == nelec and na - nb == twosz:
            idx.append(st)
    return np.asarray(idx)
