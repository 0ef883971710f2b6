"""Exact Ozaki-scheme emulation of C = A B (oracle; test infrastructure only).

Follows the paper's four steps (section "Theory of emulated FP64 arithmetic"):
 1) fixed point with one exponent shared per row of A and per column of B;
 2) split into S slices A^t, B^u of 8 bits each;
 3) every kept slice pair multiplied exactly (integers);
 4) products accumulated at high precision and converted back to FP64.
and the slice/bit relation of section "Numerical procedure": S slices hold
8S-1 magnitude bits plus the sign (S = ceildiv(bits+1, 8): 15,23,...,55 bits
for S = 2..7).  The "lower-triangular" products that are dropped are those
with t + u > S + 1 (section "Theory ...": the less significant part of the
S x S grid).

Readings fixed here (the paper is silent on them):
 * exponent: e = the smallest integer with max|a| <= (127/128) 2^e (a zero
   row has e = 0);
 * fixed point: X = RN_even(a * 2^(8S-1-e)), an integer with
   |X| <= 127*256^(S-1);
 * slices: the balanced base-256 digits of X, d_1..d_S in [-128, 127]
   (INT8), X = sum_t d_t 256^(S-t); a slice level s <= S uses d_1..d_s;
 * accumulation: the exact integer sum of the kept slice products, rounded
   ONCE to FP64 (round to nearest, ties to even).  The result is then
   independent of summation order.

Parity: pinned (tests/test_oracle_ozaki.py) by digit reconstruction, the
8S-1 bit precision, exact integer products, the closed-form error bound,
exact reproduction of small-integer matrices, power-of-two scaling and
transpose invariances, and the hand-worked fixtures in tests/golden/.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

ROW_LIMIT = Fraction(127, 128)


def exponent_of(maxabs: float) -> int:
    """Shared exponent of a row/column with largest magnitude ``maxabs``."""
    if maxabs == 0.0:
        return 0
    mant, ex = math.frexp(maxabs)          # maxabs = mant * 2^ex, mant in [0.5, 1)
    return ex if Fraction(mant) <= ROW_LIMIT else ex + 1


def row_exponents(A: np.ndarray) -> np.ndarray:
    return np.array([exponent_of(float(np.max(np.abs(r)))) if r.size else 0 for r in A], dtype=np.int64)


def fixed_point(A: np.ndarray, e: np.ndarray, S: int) -> np.ndarray:
    """X_ij = RN_even(a_ij * 2^(8S-1-e_i)) as Python ints (object array)."""
    X = np.empty(A.shape, dtype=object)
    for i in range(A.shape[0]):
        sc = Fraction(2) ** (8 * S - 1 - int(e[i]))
        for j in range(A.shape[1]):
            X[i, j] = round(Fraction(float(A[i, j])) * sc)   # Fraction.__round__ ties to even
    return X


def fixed_point_int(A: np.ndarray, e: np.ndarray, S: int) -> np.ndarray:
    """The same X_ij = RN_even(a_ij * 2^(8S-1-e_i)) as ``fixed_point``, as int64, for S <= 7
    (|X| < 2^55): a_ij = +-m 2^E with m the integer significand, so X = RN_even(m 2^(E+8S-1-e_i)),
    a left shift or a right shift rounded half to even, done on the integer m.  Equality with the
    Fraction definition is pinned in tests/test_oracle_ozaki.py."""
    if S > 7:
        raise ValueError("fixed_point_int needs S <= 7")
    A = np.asarray(A, dtype=np.float64)
    bits = A.view(np.int64)
    be = (bits >> 52) & 0x7FF
    f = bits & ((1 << 52) - 1)
    m = np.where(be > 0, f | (1 << 52), f)
    E = np.where(be > 0, be - 1075, -1074)
    sh = E + (8 * S - 1) - np.asarray(e, dtype=np.int64).reshape(-1, 1)
    X = np.zeros(A.shape, dtype=np.int64)
    left = sh >= 0
    X[left] = m[left] << sh[left]
    right = (~left) & (sh > -64)
    r = -sh[right]
    mr = m[right]
    q = mr >> r
    rem = mr - (q << r)
    half = np.int64(1) << (r - 1)
    q = q + ((rem > half) | ((rem == half) & ((q & 1) == 1))).astype(np.int64)
    X[right] = q
    return np.where(bits < 0, -X, X)


def digits(X: np.ndarray, S: int) -> list:
    """Balanced base-256 digits of every entry: list of S int64 arrays, d_1 first."""
    D = [np.zeros(X.shape, dtype=np.int64) for _ in range(S)]
    it = np.nditer(np.zeros(X.shape), flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        x = int(X[idx])
        for t in range(S - 1, -1, -1):
            d = ((x + 128) % 256) - 128
            D[t][idx] = d
            x = (x - d) // 256
        if x != 0:
            raise ValueError("fixed-point value outside the S-digit balanced range")
    return D


def digits_int(X: np.ndarray, S: int) -> list:
    """``digits`` for an int64 array X (|X| < 2^55): the same balanced base-256 digits."""
    x = np.asarray(X, dtype=np.int64).copy()
    D = [None] * S
    for t in range(S - 1, -1, -1):
        d = ((x + 128) % 256) - 128
        D[t] = d
        x = (x - d) >> 8
    if np.any(x != 0):
        raise ValueError("fixed-point value outside the S-digit balanced range")
    return D


def slice_rows(A: np.ndarray, S: int):
    """Per-row exponents and S digit planes of A (A-role operand).  S <= 7 takes the integer form
    of the fixed point and digits (``fixed_point_int``, ``digits_int``), S >= 8 the Fraction form."""
    A = np.asarray(A, dtype=np.float64)
    e = row_exponents(A)
    if S <= 7:
        return e, digits_int(fixed_point_int(A, e, S), S)
    return e, digits(fixed_point(A, e, S), S)


def slice_cols(B: np.ndarray, S: int):
    """Per-column exponents and S digit planes of B (B-role operand)."""
    e, D = slice_rows(np.asarray(B, dtype=np.float64).T, S)
    return e, [d.T.copy() for d in D]


def kept_pairs(s: int, triangle: bool = True) -> list:
    """Slice pairs (t, u), 1-based, that are multiplied: t + u <= s + 1 (triangle) or all s^2."""
    return [(t, u) for t in range(1, s + 1) for u in range(1, s + 1) if (not triangle) or t + u <= s + 1]


def slice_products(DA: list, DB: list, s: int, triangle: bool = True) -> dict:
    """Exact integer slice products P_tu = A^t B^u (int64; exact for K < 2^49)."""
    return {(t, u): DA[t - 1] @ DB[u - 1] for (t, u) in kept_pairs(s, triangle)}


def round_scaled(Z: int, k: int) -> float:
    """RN_even(Z * 2^k) as an IEEE double (one rounding, subnormals and overflow included)."""
    if Z == 0:
        return 0.0
    try:
        if k >= 0:
            return float(Z << k)
        return float(Fraction(Z, 1 << (-k)))
    except OverflowError:
        return math.copysign(math.inf, Z)


def ozaki_gemm(A, B, S: int, s: int | None = None, triangle: bool = True, alpha: float = 1.0,
               beta: float = 0.0, C=None) -> np.ndarray:
    """Emulated FP64 C = alpha * (A B) + beta * C with S-deep slicing used at level s.

    The emulated product is RN(2^(ea_i+eb_j-2(8S-1)) * sum_{(t,u) kept} 256^(2S-t-u) P_tu),
    one rounding; then alpha*c and beta*C are each rounded and added (no fused multiply-add).
    """
    s = S if s is None else s
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    ea, DA = slice_rows(A, S)
    eb, DB = slice_cols(B, S)
    P = slice_products(DA, DB, s, triangle)
    m, n = A.shape[0], B.shape[1]
    out = np.empty((m, n))
    for i in range(m):
        for j in range(n):
            Z = 0
            for (t, u), Ptu in P.items():
                Z += int(Ptu[i, j]) * (256 ** (2 * S - t - u))
            out[i, j] = round_scaled(Z, int(ea[i]) + int(eb[j]) - 2 * (8 * S - 1))
    if alpha != 1.0:
        out = alpha * out
    if beta != 0.0:
        out = out + beta * np.asarray(C, dtype=np.float64)
    return out


def error_bound(A, B, S: int, s: int | None = None, triangle: bool = True) -> np.ndarray:
    """Per-element bound on |C_emul - (AB)_ij| before the final rounding.

    With u_a = 2^(ea-(8s-1)) the unit of the s-digit fixed point, every a
    differs from its s-digit representative by at most 0.51 u_a (half a unit
    from the rounding to 8S-1 bits plus at most 128(256^(S-s)-1)/255 units of
    the dropped tail, both < 0.51 u_a); likewise b.  The truncated products
    add  sum_k (0.51 u_a |b_kj| + 0.51 u_b |a_ik| + 0.27 u_a u_b)  and the
    dropped diagonals g = t+u >= s+2 add at most
    sum_g (#pairs on g) K 2^14 2^(ea+eb+2-8g) (|d| <= 128).
    """
    s = S if s is None else s
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    ea = row_exponents(A).astype(np.float64)
    eb = row_exponents(B.T).astype(np.float64)
    K = A.shape[1]
    ua = np.ldexp(1.0, (ea - (8 * s - 1)).astype(np.int64))
    ub = np.ldexp(1.0, (eb - (8 * s - 1)).astype(np.int64))
    bound = 0.51 * ua[:, None] * np.abs(B).sum(axis=0)[None, :]
    bound += 0.51 * np.abs(A).sum(axis=1)[:, None] * ub[None, :]
    bound += 0.27 * K * ua[:, None] * ub[None, :]
    if triangle:
        drop = 0.0
        for g in range(s + 2, 2 * s + 1):
            npairs = 2 * s + 1 - g
            drop += npairs * K * 2.0 ** (14 + 2 - 8 * g)
        bound += drop * np.ldexp(1.0, (ea[:, None] + eb[None, :]).astype(np.int64))
    return bound


def ulp(x: np.ndarray) -> np.ndarray:
    x = np.abs(np.asarray(x, dtype=np.float64))
    return np.spacing(x)
