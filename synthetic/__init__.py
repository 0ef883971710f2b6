"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only *generates inputs*: integrals, sector structures, operator
blocks and trial vectors.  It holds none of the method's arithmetic (no
slicing, no products, no H_eff assembly, no eigensolver), so that the oracle
under ``oracle/`` and the CUDA path under ``paper_2510_04795_gb300/`` can both
take their inputs from here without sharing any code with each other.

Two kinds of generator are used:

* small structural data (integrals, sector dimensions, term lists) comes from
  ``numpy.random.Generator(PCG64(seed))`` on the host and is handed to both
  sides as arrays;
* bulk block values (operator blocks, psi) come from a counter-based
  generator (the SplitMix64 finaliser of Steele, Lea and Flood, 2014, applied
  to ``seed, stream, counter``), evaluated with 64-bit integer torch ops.
  Only exact integer ops and correctly rounded IEEE +,-,*,ldexp are used after
  the hash, so a block generated on a GPU is bit-identical to the same block
  generated on the host.  That lets the oracle regenerate any sampled block of
  a full-size workload on the CPU.

Distribution stand-ins (the paper's molecular integrals are not available):
"N(0,1)" is an Irwin-Hall(4) variate rescaled to unit variance, and the
exponent-spread law "N(0,1)*10^U(-6,0)" is N(0,1) * (1+u) * 2^-j with j
uniform on {0..19} and u uniform on [0,1): log10 magnitudes spread over about
six decades, and every value is exactly reproducible on any device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

__all__ = [
    "integrals", "uniform01", "normal", "block_values", "HeffStructure", "heff_structure",
    "gen_task_blocks", "gen_psi", "CONFIGS",
]

_M64 = (1 << 64) - 1


def _s64(x: int) -> int:
    """Python int (mod 2^64) -> the signed int64 with the same bit pattern."""
    x &= _M64
    return x - (1 << 64) if x >> 63 else x


_GOLD = _s64(0x9E3779B97F4A7C15)
_MIX1 = _s64(0xBF58476D1CE4E5B9)
_MIX2 = _s64(0x94D049BB133111EB)


def _srl(z: torch.Tensor, k: int) -> torch.Tensor:
    # logical right shift of int64 bit patterns
    return (z >> k) & ((1 << (64 - k)) - 1)


def _splitmix(z: torch.Tensor) -> torch.Tensor:
    z = z + _GOLD
    z = (z ^ _srl(z, 30)) * _MIX1
    z = (z ^ _srl(z, 27)) * _MIX2
    return z ^ _srl(z, 31)


def _key(seed: int, stream: int) -> int:
    # decorrelate (seed, stream) through one host-side SplitMix64 round
    z = (seed * 0x632BE59BD9B4E019 + stream * 0xD1B54A32D192ED03 + 0x8CB92BA72F3D8DD7) & _M64
    z = (z + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return _s64(z ^ (z >> 31))


# Element idx of the stream (seed, stream) draws lane l from splitmix64((8 idx + l) ^ key(seed, stream)).
def _lanes(idx: torch.Tensor, key, lane: int) -> torch.Tensor:
    return _splitmix((idx * 8 + lane) ^ key)


def _u01(bits: torch.Tensor) -> torch.Tensor:
    return _srl(bits, 11).to(torch.float64) * (2.0 ** -53)


def _values(idx: torch.Tensor, key, spread: bool, width: int = 20) -> torch.Tensor:
    s = _u01(_lanes(idx, key, 0))
    s = s + _u01(_lanes(idx, key, 1))
    s = s + _u01(_lanes(idx, key, 2))
    s = s + _u01(_lanes(idx, key, 3))
    v = (s - 2.0) * math.sqrt(3.0)
    if spread:
        j = _srl(_lanes(idx, key, 4), 11) % width  # uniform on 0..width-1 up to 2^-48
        u = _u01(_lanes(idx, key, 5))
        v = v * torch.ldexp(1.0 + u, -j.to(torch.int32))
    return v


def uniform01(seed: int, stream: int, n: int, device="cpu", lane: int = 0) -> torch.Tensor:
    """n uniforms on [0,1), k*2^-53 with k the top 53 hash bits (exact)."""
    return _u01(_lanes(torch.arange(n, dtype=torch.int64, device=device), _key(seed, stream), lane))


def normal(seed: int, stream: int, n: int, device="cpu") -> torch.Tensor:
    """Unit-variance Irwin-Hall(4) stand-in for N(0,1), bit-reproducible across devices."""
    return _values(torch.arange(n, dtype=torch.int64, device=device), _key(seed, stream), False)


def block_values(seed: int, stream: int, rows: int, cols: int, spread: bool, device="cpu",
                 width: int = 20) -> torch.Tensor:
    """A rows x cols float64 block; ``spread`` applies the exponent spread 2^-j, j uniform on
    0..width-1 (width 20: the six-decade spread)."""
    idx = torch.arange(rows * cols, dtype=torch.int64, device=device)
    return _values(idx, _key(seed, stream), spread, width).reshape(rows, cols)


# --------------------------------------------------------------------------------------------
# ab initio integrals (orbitals in index order, chemist notation, no core energy)
# --------------------------------------------------------------------------------------------

def integrals(L: int, seed: int = 0):
    """Random FP64 integrals: h_pq = h_qp ~ N(0,1) e^{-|p-q|/2};
    (pq|rs) ~ N(0, sd 0.5) e^{-(|p-q|+|r-s|)/2} with the 8-fold permutational symmetry.
    Returns (h[L,L], eri[L,L,L,L]) as numpy float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = np.zeros((L, L))
    for p in range(L):
        for q in range(p + 1):
            h[p, q] = h[q, p] = rng.normal(0.0, 1.0) * math.exp(-abs(p - q) / 2.0)
    eri = np.zeros((L, L, L, L))
    pairs = [(p, q) for p in range(L) for q in range(p + 1)]
    for a, (p, q) in enumerate(pairs):
        for (r, s) in pairs[: a + 1]:
            v = rng.normal(0.0, 0.5) * math.exp(-(abs(p - q) + abs(r - s)) / 2.0)
            for (i, j) in ((p, q), (q, p)):
                for (k, l) in ((r, s), (s, r)):
                    eri[i, j, k, l] = v
                    eri[k, l, i, j] = v
    return h, eri


# --------------------------------------------------------------------------------------------
# block-sparse two-site H_eff structure (synthetic sector layout)
# --------------------------------------------------------------------------------------------

@dataclass
class HeffStructure:
    """Sector layout of Y = sum_k c_k L_k psi R_k^T.

    Left enlarged sectors q = 0..nsec-1 carry labels (n, 2Sz); psi block q is
    m[q] x n[q] (n[q] is the dimension of the complementary right sector).
    Each task t = (term, src, dst) contributes
        Y[dst] += coef[term] * L_t (m[dst] x m[src]) @ psi[src] @ R_t^T (R_t: n[dst] x n[src]).
    Terms come in transpose pairs (2j, 2j+1): the block of term 2j+1 for
    (src=b, dst=a) is the transpose of the block of term 2j for (src=a, dst=b),
    so that H_eff is symmetric.
    """
    labels: list
    m: np.ndarray
    n: np.ndarray
    term_delta: list
    term_coef: np.ndarray
    tasks: np.ndarray            # int64 [ntask, 3] = (term, src, dst)
    spread: bool
    seed: int
    partner: np.ndarray = field(default=None)   # task index of the transpose partner
    widths: np.ndarray = field(default=None)    # per-sector spread widths (None: 20 everywhere)

    @property
    def nsec(self) -> int:
        return len(self.m)

    @property
    def ntask(self) -> int:
        return len(self.tasks)

    def flops(self) -> int:
        """FP64 flops of the native contraction: sum over tasks of 2(m'mn + m'nn')."""
        t = self.tasks
        mp, mm = self.m[t[:, 2]].astype(np.int64), self.m[t[:, 1]].astype(np.int64)
        nn, nq = self.n[t[:, 1]].astype(np.int64), self.n[t[:, 2]].astype(np.int64)
        return int(np.sum(2 * (mp * mm * nn + mp * nn * nq)))

    def psi_offsets(self) -> np.ndarray:
        sz = self.m.astype(np.int64) * self.n.astype(np.int64)
        return np.concatenate([[0], np.cumsum(sz)])


def _loguniform_int(rng, lo, hi, size):
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), size))).astype(np.int64).clip(lo, hi)


def heff_structure(grid=(8, 5), dims=(8, 256), nterms=128, spread=True, seed=1,
                   widths: bool = False) -> HeffStructure:
    """Synthetic sector structure.

    ``grid`` = (number of particle-number values, number of 2Sz values) of
    left enlarged sectors; block dims are i.i.d. log-uniform integers in
    ``dims``.  Term mix (shaped like complementary-operator H_eff): two
    Hamiltonian terms (Delta=0), then about 20% one-fermion (dN=+-1,
    d2Sz=+-1), 40% pair (dN in {+-2, 0}, d2Sz in {0, +-2}) and 40% density-like
    (Delta=0) terms, all in transpose pairs.  A task exists only where
    src + Delta is a sector of the grid.  ``widths=True`` draws a spread width w_q on 1..20 per
    sector; the blocks of a task between sectors a and b then use width (w_a + w_b) // 2, so that
    the exponent spread differs between the stacked products of different sectors.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    A, B = grid
    labels = []
    for a in range(A):
        for b in range(B):
            labels.append((a, b))  # (particle-number index, 2Sz index) on the grid
    index = {lab: i for i, lab in enumerate(labels)}
    nsec = len(labels)
    m = _loguniform_int(rng, dims[0], dims[1], nsec)
    n = _loguniform_int(rng, dims[0], dims[1], nsec)
    npair = max(1, nterms // 2)
    deltas, coefs = [], []
    one = [(1, 1), (1, -1)]
    pair = [(2, 0), (2, 2), (2, -2), (0, 2)]
    for j in range(npair):
        if j == 0:
            d = (0, 0)
        else:
            x = rng.uniform()
            if x < 0.2:
                d = one[rng.integers(len(one))]
            elif x < 0.6:
                d = pair[rng.integers(len(pair))]
            else:
                d = (0, 0)
            if d != (0, 0) and rng.uniform() < 0.5:
                d = (-d[0], -d[1])
        c = 1.0 if j == 0 else float(rng.uniform(0.5, 1.5))
        deltas += [d, (-d[0], -d[1])]
        coefs += [c, c]
    tasks, partner_key = [], []
    for k in range(len(deltas)):
        dn, ds = deltas[k]
        for q, (a, b) in enumerate(labels):
            tgt = index.get((a + dn, b + ds))
            if tgt is not None:
                tasks.append((k, q, tgt))
    tasks = np.asarray(tasks, dtype=np.int64).reshape(-1, 3)
    pos = {(int(k), int(s), int(d)): i for i, (k, s, d) in enumerate(tasks)}
    partner = np.empty(len(tasks), dtype=np.int64)
    for i, (k, s, d) in enumerate(tasks):
        partner[i] = pos[(int(k) ^ 1, int(d), int(s))]
    w = rng.integers(1, 21, size=nsec) if widths else None
    return HeffStructure(labels, m, n, deltas, np.asarray(coefs), tasks, spread, seed, partner, w)


def _task_stream(st: HeffStructure, t: int, side: int) -> int:
    # the even member of a transpose pair owns the values; the odd one is its transpose
    k, s, d = (int(x) for x in st.tasks[t])
    if k % 2 == 1:
        k, s, d = k ^ 1, d, s
    return ((k * 4096 + s) * 4096 + d) * 2 + side


def gen_task_blocks(st: HeffStructure, t: int, value_seed: int = 2, device="cpu"):
    """(L_t, R_t) for task t as float64 tensors of shape (m[dst], m[src]) and (n[dst], n[src])."""
    k, s, d = (int(x) for x in st.tasks[t])
    odd = k % 2 == 1
    if odd:
        s, d = d, s
    w = 20 if st.widths is None else int(st.widths[s] + st.widths[d]) // 2
    Lb = block_values(value_seed, _task_stream(st, t, 0), int(st.m[d]), int(st.m[s]), st.spread, device, w)
    Rb = block_values(value_seed, _task_stream(st, t, 1), int(st.n[d]), int(st.n[s]), st.spread, device, w)
    if odd:
        Lb, Rb = Lb.T.contiguous(), Rb.T.contiguous()
    return Lb, Rb


def gen_all_task_blocks(st: HeffStructure, value_seed: int = 2, device="cuda", chunk: int = 1 << 27):
    """All (L_t, R_t) blocks, generated in large batches (bit-identical to gen_task_blocks).

    Returns (Lbuf, Rbuf, Loff, Roff): flat float64 buffers and per-task element offsets; task t's
    L block is Lbuf[Loff[t]:Loff[t]+m[dst]*m[src]].view(m[dst], m[src]) (likewise R with n)."""
    if st.widths is not None:
        raise ValueError("per-sector spread widths: use gen_task_blocks")
    t = st.tasks
    mdst, msrc = st.m[t[:, 2]].astype(np.int64), st.m[t[:, 1]].astype(np.int64)
    ndst, nsrc = st.n[t[:, 2]].astype(np.int64), st.n[t[:, 1]].astype(np.int64)
    out = []
    for side, (r, c) in enumerate(((mdst, msrc), (ndst, nsrc))):
        sizes = r * c
        off = np.concatenate([[0], np.cumsum(sizes)])
        buf = torch.empty(int(off[-1]), dtype=torch.float64, device=device)
        owners = np.nonzero(t[:, 0] % 2 == 0)[0]
        keys = np.array([_key(value_seed, _task_stream(st, int(i), side)) for i in owners], dtype=np.int64)
        # batches of owner tasks with about `chunk` elements each
        start = 0
        while start < len(owners):
            tot, end = 0, start
            while end < len(owners) and (tot == 0 or tot + sizes[owners[end]] <= chunk):
                tot += int(sizes[owners[end]])
                end += 1
            sel = owners[start:end]
            sz = torch.as_tensor(sizes[sel], device=device)
            kk = torch.as_tensor(keys[start:end], device=device)
            which = torch.repeat_interleave(torch.arange(len(sel), device=device), sz)
            first = torch.cumsum(sz, 0) - sz
            local = torch.arange(tot, dtype=torch.int64, device=device) - first[which]
            vals = _values(local, kk[which], st.spread)
            pos = 0
            for i, ti in enumerate(sel):
                n_ = int(sizes[ti])
                buf[off[ti]:off[ti] + n_].copy_(vals[pos:pos + n_])
                pos += n_
            del vals, local, which
            start = end
        # partners are transposes of their owner's block
        for ti in np.nonzero(t[:, 0] % 2 == 1)[0]:
            p = int(st.partner[ti])
            src = buf[off[p]:off[p] + sizes[p]].view(int(r[p]), int(c[p]))
            buf[off[ti]:off[ti] + sizes[ti]].view(int(r[ti]), int(c[ti])).copy_(src.T)
        out += [buf, off]
    return out[0], out[2], out[1], out[3]


def gen_psi(st: HeffStructure, seed: int = 3, device="cpu", decades: float = 0.0) -> torch.Tensor:
    """psi as one flat float64 vector (blocks q = 0.. concatenated, each row-major).

    ``decades`` > 0 scales block q by 2^-round(decades log2(10) u_q), u_q uniform on [0, 1): sector
    weights spread over that many decades, as the quantum-number sectors of a DMRG wavefunction."""
    off = st.psi_offsets()
    v = normal(seed, 1 << 40, int(off[-1]), device)
    # scale by a power of two so that |psi| is about 1 (exact on every device)
    e = -int(round(0.5 * math.log2(max(1, int(off[-1])))))
    v = torch.ldexp(v, torch.tensor(e, dtype=torch.int32, device=device))
    if decades > 0.0:
        u = uniform01(seed, (1 << 40) + 1, st.nsec).numpy()
        for q in range(st.nsec):
            k = -int(round(decades * math.log2(10.0) * float(u[q])))
            v[off[q]:off[q + 1]] = torch.ldexp(v[off[q]:off[q + 1]], torch.tensor(k, dtype=torch.int32, device=device))
    return v


# Workload shapes named after what they are (block count, sizes, terms).
CONFIGS = {
    # single H_eff*psi, 40 blocks of 8..256, exponent spread, slice count swept
    "heff40_8-256": dict(grid=(8, 5), dims=(8, 256), nterms=128, spread=True),
    # batched uneven sector GEMMs, 300 blocks of 16..1024, about 200 terms, N(0,1) entries
    "heff300_16-1024": dict(grid=(20, 15), dims=(16, 1024), nterms=200, spread=False),
}
