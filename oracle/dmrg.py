"""Explicit-basis two-site DMRG (oracle; test infrastructure only).

The paper's DMRG sweeps over the chain, solves the two-site eigenproblem of the effective
Hamiltonian with a Krylov method and truncates with an SVD of the two-site tensor (section
"Theory of TNS/DMRG regarding error analysis"; the energy approaches the exact ground state from
above).  This module is the formalism-free definition of one such sweep: every block basis is kept
as explicit vectors in the Fock space of its orbitals, and the effective Hamiltonian of a bond is
literally P^T H P, with H the full CI Hamiltonian and P the embedding of the two-site product basis
(left block (x) site i (x) site i+1 (x) right block) into the determinant basis.  Nothing here
uses operators of blocks, so it pins the renormalised-operator construction of the library.

Conventions (readings where the paper is silent):
 * Determinants are orbital-major occupation patterns: bit 2p is orbital p spin up, bit 2p+1 spin
   down, and |pattern> = prod_x (a^+_x)^{n_x} |0> in ascending x.  A product of left, site and right
   patterns is then the determinant itself (no sign), because every part lists its orbitals in
   the global order.
 * Site states are 0 = |0>, 1 = |up>, 2 = |down>, 3 = |up down>, i.e. the two bits of the orbital.
 * Start: every right block is the single state given by the reference determinant (orbitals
   filled from 0: n_up = (N + 2Sz)/2 up electrons, n_down = (N - 2Sz)/2 down electrons).
 * A sweep is a left-to-right half-sweep over bonds 0..L-2 followed by a right-to-left one over
   bonds L-2..0; every bond solves for the lowest eigenpair (the energy is recorded) and every
   bond but the last of a half-sweep truncates.
 * Truncation of the enlarged block (block (x) site): if it has at most D product states, keep
   them all (no rotation).  Otherwise take the eigenpairs of the reduced density matrix of each
   quantum-number sector (rho = psi psi^T on the left, psi^T psi on the right; its eigenvalues are
   the squared singular values), keep the largest ones above 1e-14, at most D of them, and never
   cut through a group of equal eigenvalues (those within 1e-12 lambda_max + 1e-8 lambda at the
   cut, e.g. members of a spin multiplet): the whole group is dropped instead.
 * Emulated density matrices (the paper's truncation-precision study, same section): with
   ``rdm = (S, s)`` every rho is the emulated product of ``ozaki.ozaki_gemm`` instead of FP64.
Parity: pinned (tests/test_oracle_dmrg.py) by FCI: without truncation the sweep energy equals
the FCI energy, with truncation it stays above it and decreases sweep by sweep; with emulated
density matrices at S = 7 (noise far below the keep threshold) the sweep is the FP64 one.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fci, ozaki

SITE_Q = [(0, 0), (1, 1), (1, -1), (2, 0)]   # (electrons, 2 Sz) of the site states 0..3
LAMBDA_MIN = 1e-14


def orbital_major_hamiltonian(h, eri, nelec: int, twosz: int):
    """(H, patterns): the FCI Hamiltonian of the sector (nelec, twosz) in the orbital-major
    determinant basis (ordered as the alpha-string x beta-string product basis of ``fci``), and
    the occupation pattern of every basis state.  H_om = D H_af D, D the sign that reorders
    prod_{alpha} a^+ prod_{beta} a^+ into orbital-major order."""
    L = h.shape[0]
    na, nb = (nelec + twosz) // 2, (nelec - twosz) // 2
    Haf = fci.hamiltonian(h, eri, na, nb)
    sa, sb = fci.strings(L, na), fci.strings(L, nb)
    pats = np.zeros(len(sa) * len(sb), dtype=np.int64)
    sgn = np.zeros(len(sa) * len(sb))
    for i, a in enumerate(sa):
        for j, b in enumerate(sb):
            pat, inv = 0, 0
            for p in range(L):
                if (a >> p) & 1:
                    pat |= 1 << (2 * p)
                    # beta electrons on lower orbitals must pass this alpha creator
                    inv += bin(b & ((1 << p) - 1)).count("1")
                if (b >> p) & 1:
                    pat |= 1 << (2 * p + 1)
            pats[i * len(sb) + j] = pat
            sgn[i * len(sb) + j] = -1.0 if inv % 2 else 1.0
    D = sp.diags(sgn)
    return (D @ Haf @ D).tocsr(), pats


class _Sector:
    """Explicit block sector: patterns (global bit patterns of the block's orbitals) and U, whose
    columns are the block states as vectors over those patterns."""

    def __init__(self, q, patterns, U):
        self.q = q
        self.patterns = np.asarray(patterns, dtype=np.int64)
        self.U = np.asarray(U, dtype=np.float64)

    @property
    def k(self):
        return self.U.shape[1]


def _qadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def _enlarge(block: dict, site: int, site_first: bool) -> dict:
    """Product basis of block (x) site (site_first=False) or site (x) block (True), grouped by
    quantum number: each sector's patterns and a block-diagonal U (one block per piece)."""
    pieces = {}
    for s in range(4):
        for q, sec in block.items():
            qn = _qadd(q, SITE_Q[s])
            pieces.setdefault(qn, []).append((sec.patterns | (s << (2 * site)), sec.U))
    out = {}
    for qn, lst in pieces.items():
        npat = sum(len(p) for p, _ in lst)
        k = sum(U.shape[1] for _, U in lst)
        pats = np.concatenate([p for p, _ in lst])
        U = np.zeros((npat, k))
        r = c = 0
        for p, Ub in lst:
            U[r:r + len(p), c:c + Ub.shape[1]] = Ub
            r += len(p)
            c += Ub.shape[1]
        out[qn] = _Sector(qn, pats, U)
    return out


def select_kept(lams: list, D: int) -> int:
    """Number of eigenvalues kept from the descending list ``lams``: at most D, all above
    LAMBDA_MIN, never cutting through a group of equal values."""
    cand = [x for x in lams if x > LAMBDA_MIN]
    k = min(D, len(cand))
    lmax = cand[0] if cand else 0.0
    while 0 < k < len(cand) and cand[k - 1] - cand[k] <= 1e-12 * lmax + 1e-8 * cand[k - 1]:
        k -= 1
    return k


def _truncate(enl: dict, psi_blocks: dict, D: int, left: bool, rdm=None) -> dict:
    """New block from the enlarged block ``enl`` and the two-site blocks psi_blocks[q] (rows: the
    enlarged sector q of the left side; columns: the right side), by the rule of the header.
    ``rdm = (S, s)`` forms every density matrix as the emulated product of ``ozaki.ozaki_gemm``
    (S slices used at level s) instead of in FP64; the eigendecomposition stays FP64."""
    total = sum(sec.k for sec in enl.values())
    if total <= D:
        return enl
    eig = {}
    allv = []
    for q, sec in enl.items():
        M = psi_blocks.get(q)
        if M is None or M.size == 0:
            continue
        if rdm is None:
            rho = M @ M.T if left else M.T @ M
        else:
            rho = ozaki.ozaki_gemm(M, M.T, rdm[0], rdm[1]) if left else ozaki.ozaki_gemm(M.T, M, rdm[0], rdm[1])
        w, V = np.linalg.eigh(0.5 * (rho + rho.T))
        w, V = w[::-1], V[:, ::-1]
        eig[q] = (w, V)
        allv.extend(float(x) for x in w)
    allv.sort(reverse=True)
    k = select_kept(allv, D)
    if k == 0:
        raise RuntimeError("truncation kept no state")
    cut = allv[k - 1]
    out = {}
    for q, (w, V) in eig.items():
        keep = w >= cut
        if np.any(keep):
            sec = enl[q]
            out[q] = _Sector(q, sec.patterns, sec.U @ V[:, keep])
    assert sum(s.k for s in out.values()) == k
    return out


def _reference_blocks(L, nelec, twosz):
    """Right blocks of the start: block j (orbitals j..L-1) holds the reference determinant's
    part on those orbitals (one state)."""
    na, nb = (nelec + twosz) // 2, (nelec - twosz) // 2
    ref = 0
    for p in range(na):
        ref |= 1 << (2 * p)
    for p in range(nb):
        ref |= 1 << (2 * p + 1)
    blocks = {}
    for j in range(L + 1):
        mask = sum(3 << (2 * p) for p in range(j, L))
        pat = ref & mask
        n = bin(pat).count("1")
        nup = bin(pat & sum(1 << (2 * p) for p in range(L))).count("1")
        q = (n, nup - (n - nup))
        blocks[j] = {q: _Sector(q, [pat], np.ones((1, 1)))}
    return blocks


class ExplicitDMRG:
    """Two-site DMRG with explicit block bases (see the module header)."""

    def __init__(self, h, eri, nelec: int, twosz: int, D: int, eig_tol: float = 1e-13, rdm=None):
        self.L = h.shape[0]
        self.N, self.twosz, self.D = nelec, twosz, D
        self.H, pats = orbital_major_hamiltonian(h, eri, nelec, twosz)
        self.index = np.full(1 << (2 * self.L), -1, dtype=np.int64)
        self.index[pats] = np.arange(len(pats))
        self.target = (nelec, twosz)
        self.eig_tol = eig_tol
        self.rdm = rdm          # None (FP64 density matrices) or (S, s) for emulated ones
        vac = {(0, 0): _Sector((0, 0), [0], np.ones((1, 1)))}
        self.left = {0: vac}                       # left[i]: block of orbitals 0..i-1
        self.right = _reference_blocks(self.L, nelec, twosz)   # right[j]: orbitals j..L-1
        self.energies = []

    def _solve(self, i):
        """Lowest eigenpair of P^T H P at bond (i, i+1); returns (E, psi blocks by LE sector)."""
        LE = _enlarge(self.left[i], i, site_first=False)
        RE = _enlarge(self.right[i + 2], i + 1, site_first=True)
        secs = [(q, LE[q], RE[(self.target[0] - q[0], self.target[1] - q[1])]) for q in LE
                if (self.target[0] - q[0], self.target[1] - q[1]) in RE]
        ncol = sum(a.k * b.k for _, a, b in secs)
        P = np.zeros((self.H.shape[0], ncol))
        off = 0
        for q, a, b in secs:
            idx = self.index[(a.patterns[:, None] | b.patterns[None, :]).ravel()]
            assert np.all(idx >= 0)
            P[idx, off:off + a.k * b.k] += np.kron(a.U, b.U)
            off += a.k * b.k
        if ncol <= 600:
            Heff = P.T @ (self.H @ P)
            w, V = np.linalg.eigh(0.5 * (Heff + Heff.T))
            E, x = float(w[0]), V[:, 0]
        else:
            op = spla.LinearOperator((ncol, ncol), matvec=lambda v: P.T @ (self.H @ (P @ v)), dtype=np.float64)
            w, V = spla.eigsh(op, k=1, which="SA", tol=self.eig_tol, v0=np.ones(ncol))
            E, x = float(w[0]), V[:, 0]
        blocks, off = {}, 0
        for q, a, b in secs:
            blocks[q] = x[off:off + a.k * b.k].reshape(a.k, b.k)
            off += a.k * b.k
        return E, blocks, LE, RE, P

    def sweep(self, nsweeps: int):
        L = self.L
        for _ in range(nsweeps):
            for i in range(0, L - 1):
                E, blocks, LE, RE, _ = self._solve(i)
                self.energies.append(E)
                if i < L - 2:
                    self.left[i + 1] = _truncate(LE, blocks, self.D, left=True, rdm=self.rdm)
            for i in range(L - 2, -1, -1):
                E, blocks, LE, RE, _ = self._solve(i)
                self.energies.append(E)
                if i > 0:
                    rblocks = {(self.target[0] - q[0], self.target[1] - q[1]): M for q, M in blocks.items()}
                    self.right[i + 1] = _truncate(RE, rblocks, self.D, left=False, rdm=self.rdm)
        return self.energies
