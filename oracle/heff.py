"""Block-sparse two-site effective-Hamiltonian product (oracle; test infrastructure only).

The DMRG update diagonalises H_eff on the two-site space with a Krylov solver
(section "Theory of TNS/DMRG regarding error analysis": the second
subroutine), and its matrix-vector product is built from binary tensor
contractions done as matrix multiplications (same section, first
subroutine).  With H_eff = sum_k c_k L_k (x) R_k acting on psi viewed as a
(left enlarged) x (right enlarged) matrix, the product is
    Y = sum_k c_k L_k psi R_k^T,
and with U(1)xU(1) sector symmetry every factor is block sparse: the task
(k, src, dst) adds c_k L_k[dst<-src] psi[src] R_k[dst<-src]^T to Y[dst].

Functions:
 * heff_apply_fp64     plain FP64, one numpy product per block (the error reference).
 * heff_dense          the dense matrix sum_k c_k L_k (x) R_k on vec(psi), brute force
                       (pins heff_apply_fp64 on tiny layouts).
 * heff_diag           its diagonal (the Davidson preconditioner), pinned by heff_dense.
 * heff_apply_emulated the two-stage emulated definition: for every source sector
                       one Ozaki product of the stacked L blocks with psi[src]; for
                       every target sector one Ozaki product of the concatenated
                       intermediates with the stacked (c_k R_k)^T.  Each stage is one
                       exact emulated GEMM rounded once (see ``ozaki``).
 * heff_entries_emulated  single entries of heff_apply_emulated from the operand rows they
                       depend on (for sampled checks of products too large for the
                       whole definition).

Parity: heff_apply_fp64 pinned by heff_dense (brute force) and Hermiticity;
heff_apply_emulated pinned through ``ozaki`` and by its distance to
heff_apply_fp64 staying inside the summed per-GEMM error bounds;
heff_entries_emulated pinned entry by entry against heff_apply_emulated.
"""
from __future__ import annotations

import numpy as np

from . import ozaki


def _blocks(psi_flat, st):
    off = st.psi_offsets()
    return [np.asarray(psi_flat[off[q]:off[q + 1]], dtype=np.float64).reshape(int(st.m[q]), int(st.n[q]))
            for q in range(st.nsec)]


def _flat(blocks):
    return np.concatenate([b.reshape(-1) for b in blocks]) if blocks else np.zeros(0)


def heff_apply_fp64(st, Lb: list, Rb: list, psi_flat) -> np.ndarray:
    """Y = sum over tasks of c_k (L_t psi[src]) R_t^T, FP64, blocks row-major, flat."""
    P = _blocks(psi_flat, st)
    Y = [np.zeros((int(st.m[q]), int(st.n[q]))) for q in range(st.nsec)]
    for t, (k, s, d) in enumerate(st.tasks):
        Y[d] += st.term_coef[k] * ((Lb[t] @ P[s]) @ Rb[t].T)
    return _flat(Y)


def heff_dense(st, Lb: list, Rb: list) -> np.ndarray:
    """Dense H_eff with H[(d,i,j),(s,a,b)] = sum_k c_k L[i,a] R[j,b] (Kronecker brute force)."""
    off = st.psi_offsets()
    N = int(off[-1])
    H = np.zeros((N, N))
    for t, (k, s, d) in enumerate(st.tasks):
        blk = st.term_coef[k] * np.kron(Lb[t], Rb[t])    # rows (i,j), cols (a,b), row-major pairs
        H[off[d]:off[d + 1], off[s]:off[s + 1]] += blk
    return H


def heff_diag(st, Lb: list, Rb: list) -> np.ndarray:
    """Diagonal of H_eff: element (q, i, j) gets c_k L[i, i] R[j, j] from every task with
    src == dst == q (a task with src != dst has no diagonal entries).  Pinned by the diagonal of
    heff_dense on tiny layouts."""
    off = st.psi_offsets()
    out = np.zeros(int(off[-1]))
    for t, (k, s, d) in enumerate(st.tasks):
        if s != d:
            continue
        blk = st.term_coef[k] * np.outer(np.diag(Lb[t]), np.diag(Rb[t]))
        out[off[s]:off[s + 1]] += blk.reshape(-1)
    return out


def emulated_groups(st):
    """Task order used by the two emulated stages: tasks grouped by source, then by target
    (ascending task index inside each group).  Exact integer accumulation makes the result
    independent of this order; it only fixes where each block sits in the stacked operands."""
    by_src = [[] for _ in range(st.nsec)]
    by_dst = [[] for _ in range(st.nsec)]
    for t, (k, s, d) in enumerate(st.tasks):
        by_src[s].append(t)
        by_dst[d].append(t)
    return by_src, by_dst


def heff_apply_emulated(st, Lb: list, Rb: list, psi_flat, S: int, s: int | None = None, s1=None,
                        s2=None) -> np.ndarray:
    """Two-stage emulated H_eff psi.

    Stage 1 (per source q): T = ozaki([L_t1; L_t2; ...], psi[q]) -> T_t blocks.
    Stage 2 (per target q'): Y[q'] = ozaki([T_t1 T_t2 ...], [(c R_t1)^T; (c R_t2)^T; ...]),
    where c R is rounded to FP64 first.  Both are one emulated DGEMM each (shared row
    exponents of the concatenated rows, shared column exponents of the stacked columns).
    Slice levels: s for every product, or per sector -- s1[q] for the stage-1 product of source
    sector q and s2[q] for the stage-2 product of target sector q (the precision dial per block).
    """
    s = S if s is None else s
    s1 = [s] * st.nsec if s1 is None else list(s1)
    s2 = [s] * st.nsec if s2 is None else list(s2)
    P = _blocks(psi_flat, st)
    by_src, by_dst = emulated_groups(st)
    T = [None] * st.ntask
    for q in range(st.nsec):
        ts = by_src[q]
        if not ts:
            continue
        A1 = np.vstack([Lb[t] for t in ts])
        C1 = ozaki.ozaki_gemm(A1, P[q], S, s1[q])
        r = 0
        for t in ts:
            h = Lb[t].shape[0]
            T[t] = C1[r:r + h]
            r += h
    Y = []
    for q in range(st.nsec):
        ts = by_dst[q]
        if not ts:
            Y.append(np.zeros((int(st.m[q]), int(st.n[q]))))
            continue
        A2 = np.hstack([T[t] for t in ts])
        B2 = np.vstack([(st.term_coef[st.tasks[t][0]] * Rb[t]).T for t in ts])
        Y.append(ozaki.ozaki_gemm(A2, B2, S, s2[q]))
    return _flat(Y)


def _row_times_sliced(a_row, eb, DB, S: int) -> np.ndarray:
    """ozaki_gemm(a_row[None, :], B, S) for a B given by its column slicing (eb, DB) = slice_cols(B, S):
    the same exponent rule, digits, kept pairs and single rounding as ``ozaki.ozaki_gemm``."""
    ea, DA = ozaki.slice_rows(np.asarray(a_row, dtype=np.float64)[None, :], S)
    P = ozaki.slice_products(DA, DB, S)
    out = np.empty(DB[0].shape[1])
    for j in range(out.size):
        Z = 0
        for (t, u), Ptu in P.items():
            Z += int(Ptu[0, j]) * (256 ** (2 * S - t - u))
        out[j] = ozaki.round_scaled(Z, int(ea[0]) + int(eb[j]) - 2 * (8 * S - 1))
    return out


def heff_entries_emulated(st, q: int, i: int, js, L_rows: dict, R_rows: dict, P_src: dict, S: int) -> np.ndarray:
    """Entries Y[q][i, j], j in js, of heff_apply_emulated, from one row of every operand they need.

    In an emulated product every row depends only on its own row of A (its own exponent) and on all
    of B, and every entry only on its row of A and its column of B.  Hence, with the tasks t into q,
        T_t[i, :]  = ozaki_gemm(L_t[i:i+1, :], psi[src_t])                              (stage 1)
        Y[q][i, j] = ozaki_gemm([T_t[i, :] ...], [(c_t R_t[j, :])^T ; ...])              (stage 2)
    are the numbers of the stacked products, whatever the order of the tasks (exact sums, maxima).
    L_rows[t] = row i of L_t; R_rows[t] = R_t[js, :] (one row per requested j); P_src[s] = psi block
    of source sector s.  Pinned against heff_apply_emulated entry by entry on small layouts.
    """
    js = list(js)
    tasks = [t for t in range(st.ntask) if int(st.tasks[t][2]) == q]
    sliced = {}
    a2, b2 = [], []
    for t in tasks:
        k, src = int(st.tasks[t][0]), int(st.tasks[t][1])
        if src not in sliced:
            sliced[src] = ozaki.slice_cols(np.asarray(P_src[src], dtype=np.float64), S)
        eb, DB = sliced[src]
        a2.append(_row_times_sliced(L_rows[t], eb, DB, S))
        b2.append((st.term_coef[k] * np.asarray(R_rows[t], dtype=np.float64)).T)
    if not tasks:
        return np.zeros(len(js))
    A2 = np.concatenate(a2)[None, :]
    B2 = np.vstack(b2)
    return ozaki.ozaki_gemm(A2, B2, S)[0]


def rel_frobenius(y, yref) -> float:
    y = np.asarray(y, dtype=np.float64)
    yref = np.asarray(yref, dtype=np.float64)
    return float(np.linalg.norm(y - yref) / np.linalg.norm(yref))
