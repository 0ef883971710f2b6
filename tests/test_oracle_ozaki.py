"""Pins of the exact Ozaki oracle against facts that do not come from the oracle itself."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki

GOLD = os.path.join(os.path.dirname(__file__), "golden", "slices_worked.txt")


def _golden():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v, S, e, d = [x.strip() for x in line.split("|")]
        rows.append((float(Fraction(v)), int(S), int(e), [int(x) for x in d.split()]))
    return rows


@pytest.mark.parametrize("row", _golden())
def test_hand_worked_slices(row):
    a, S, e, d = row
    ee, D = ozaki.slice_rows(np.array([[a]]), S)
    assert int(ee[0]) == e
    assert [int(Dt[0, 0]) for Dt in D] == d


def test_paper_mantissa_bits_per_slice_count():
    # section "Numerical procedure": S = ceildiv(bits+1, 8) gives 15,23,31,39,47,55 bits for S = 2..7
    bits = {S: 8 * S - 1 for S in range(2, 8)}
    assert [bits[S] for S in range(2, 8)] == [15, 23, 31, 39, 47, 55]
    for S, b in bits.items():
        assert math.ceil((b + 1) / 8) == S
    rng = np.random.default_rng(7)
    for S in range(2, 8):
        b = 8 * S - 1
        # numbers of the form k*2^-b with |k| < 2^b (b bits) in (-127/128, 127/128): exact
        k = rng.integers(-(1 << (b - 1)), 1 << (b - 1), size=32)
        a = np.array([float(Fraction(int(x), 1 << b)) for x in k])[None, :]
        a[0, 0] = 0.9  # fixes e = 0 for the whole row
        e, D = ozaki.slice_rows(a, S)
        assert e[0] == 0
        X = sum(D[t].astype(object) * 256 ** (S - 1 - t) for t in range(S))
        rec = np.array([float(Fraction(int(x), 1 << b)) for x in X[0]])
        assert np.array_equal(rec[1:], a[0, 1:])
        # one more bit than 8S-1 is not representable: the error is exactly half a unit
        odd = float(Fraction(2 * 12345 + 1, 1 << (b + 1)))
        e2, D2 = ozaki.slice_rows(np.array([[0.9, odd]]), S)
        X2 = sum(int(D2[t][0, 1]) * 256 ** (S - 1 - t) for t in range(S))
        assert abs(Fraction(X2, 1 << b) - Fraction(odd)) == Fraction(1, 1 << (b + 1))


def test_digit_ranges_and_reconstruction():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(9, 13)) * 10.0 ** rng.uniform(-6, 0, size=(9, 13))
    A[3] = 0.0
    for S in (1, 2, 3, 5, 7, 9):
        e, D = ozaki.slice_rows(A, S)
        for Dt in D:
            assert Dt.min() >= -128 and Dt.max() <= 127
        X = sum(D[t].astype(object) * 256 ** (S - 1 - t) for t in range(S))
        for i in range(A.shape[0]):
            mx = np.max(np.abs(A[i]))
            if mx == 0:
                assert e[i] == 0 and all(int(x) == 0 for x in X[i])
                continue
            assert Fraction(mx) <= Fraction(127, 128) * Fraction(2) ** int(e[i])
            assert Fraction(mx) > Fraction(127, 128) * Fraction(2) ** (int(e[i]) - 1)
            for j in range(A.shape[1]):
                err = abs(Fraction(int(X[i, j])) * Fraction(2) ** (int(e[i]) - (8 * S - 1)) - Fraction(float(A[i, j])))
                assert err <= Fraction(2) ** (int(e[i]) - 8 * S)


def test_product_counts_triangle():
    # section "Theory ...": seven slices -> 7x7 = 49 products; dropping the lower triangle keeps 28
    assert len(ozaki.kept_pairs(7, triangle=False)) == 49
    assert len(ozaki.kept_pairs(7, triangle=True)) == 28
    assert [len(ozaki.kept_pairs(s)) for s in range(3, 10)] == [6, 10, 15, 21, 28, 36, 45]


def test_slice_products_exact_integers():
    rng = np.random.default_rng(1)
    A = rng.normal(size=(5, 17))
    B = rng.normal(size=(17, 6))
    _, DA = ozaki.slice_rows(A, 4)
    _, DB = ozaki.slice_cols(B, 4)
    P = ozaki.slice_products(DA, DB, 4)
    for (t, u), Ptu in P.items():
        # brute force with Python integers
        for i in range(5):
            for j in range(6):
                assert int(Ptu[i, j]) == sum(int(DA[t - 1][i, k]) * int(DB[u - 1][k, j]) for k in range(17))


def test_integer_matrices_exact():
    # integer entries of < 2^20 are exactly representable with S >= 3 (23 bits) and the
    # product is an integer of < 2^53 -> the emulation returns it exactly
    rng = np.random.default_rng(2)
    A = rng.integers(-(1 << 19), 1 << 19, size=(7, 11)).astype(np.float64)
    B = rng.integers(-(1 << 19), 1 << 19, size=(11, 5)).astype(np.float64)
    for S in (3, 4, 7):
        C = ozaki.ozaki_gemm(A, B, S, triangle=False)
        exact = (A.astype(object) @ B.astype(object)).astype(np.float64)
        assert np.array_equal(C, exact)
    # with the triangle the dropped products are below the integer unit only for S large enough
    assert np.array_equal(ozaki.ozaki_gemm(A, B, 7), (A.astype(object) @ B.astype(object)).astype(np.float64))


def test_error_bound_and_decay():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(12, 40)) * 10.0 ** rng.uniform(-6, 0, size=(12, 40))
    B = rng.normal(size=(40, 9)) * 10.0 ** rng.uniform(-6, 0, size=(40, 9))
    exact = np.array([[float(sum(Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(40)))
                       for j in range(9)] for i in range(12)])
    errs = []
    for S in range(2, 10):
        C = ozaki.ozaki_gemm(A, B, S)
        bnd = ozaki.error_bound(A, B, S)
        err = np.abs(C - exact)
        assert np.all(err <= bnd + ozaki.ulp(exact) + ozaki.ulp(C))
        errs.append(np.max(err / np.abs(exact).max()))
    # error falls by orders of magnitude per slice until FP64 is reached
    for a, b in zip(errs[:4], errs[1:5]):
        assert b < a / 50
    assert errs[-1] < 1e-15


def test_power_of_two_scaling_and_transpose_invariance():
    rng = np.random.default_rng(4)
    A = rng.normal(size=(6, 10))
    B = rng.normal(size=(10, 7))
    S = 5
    C = ozaki.ozaki_gemm(A, B, S)
    rs = rng.integers(-30, 30, size=6)
    cs = rng.integers(-30, 30, size=7)
    C2 = ozaki.ozaki_gemm(np.ldexp(A, rs[:, None]), np.ldexp(B, cs[None, :]), S)
    assert np.array_equal(C2, np.ldexp(C, rs[:, None] + cs[None, :]))
    Ct = ozaki.ozaki_gemm(B.T, A.T, S)
    assert np.array_equal(Ct, C.T)


def test_one_rounding_against_fraction():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(3, 8))
    B = rng.normal(size=(8, 4))
    S = 6
    ea, DA = ozaki.slice_rows(A, S)
    eb, DB = ozaki.slice_cols(B, S)
    C = ozaki.ozaki_gemm(A, B, S)
    for i in range(3):
        for j in range(4):
            tot = Fraction(0)
            for (t, u) in ozaki.kept_pairs(S):
                p = sum(int(DA[t - 1][i, k]) * int(DB[u - 1][k, j]) for k in range(8))
                tot += Fraction(p) * Fraction(2) ** (int(ea[i]) + int(eb[j]) + 2 - 8 * (t + u))
            assert C[i, j] == float(tot)


def test_round_scaled_subnormal_and_overflow():
    assert ozaki.round_scaled(1, -1074) == 5e-324
    assert ozaki.round_scaled(1, -1075) == 0.0          # exactly half the smallest subnormal: ties to even -> 0
    assert ozaki.round_scaled(3, -1075) == 1e-323       # 1.5 ulp -> 2 ulp
    assert ozaki.round_scaled(1, 1024) == math.inf
    assert ozaki.round_scaled(-((1 << 53) + 1), 0) == -float(1 << 53)
    assert ozaki.round_scaled((1 << 53) + 3, 0) == float((1 << 53) + 4)


def test_alpha_beta():
    rng = np.random.default_rng(6)
    A, B, C0 = rng.normal(size=(4, 5)), rng.normal(size=(5, 3)), rng.normal(size=(4, 3))
    C = ozaki.ozaki_gemm(A, B, 7)
    out = ozaki.ozaki_gemm(A, B, 7, alpha=-0.5, beta=2.0, C=C0)
    assert np.array_equal(out, (-0.5 * C) + (2.0 * C0))


@pytest.mark.parametrize("S", [1, 2, 3, 5, 7])
def test_integer_fixed_point_equals_fraction_definition(S):
    # the int64 form used for S <= 7 against the Fraction form of the same definition: random
    # magnitudes over 40 binades, exact halfway cases of the rounding, subnormals, zeros, signs
    rng = np.random.default_rng(100 + S)
    A = rng.normal(size=(12, 40)) * np.ldexp(1.0, rng.integers(-20, 20, size=(12, 40)))
    A[0, :8] = 0.0
    A[1, :] = np.ldexp(rng.integers(1, 2 ** 20, size=40).astype(np.float64), -1074)    # subnormal row
    A[2, :] = [(k + 0.5) * 2.0 ** -(8 * S - 1) for k in range(-20, 20)]               # ties at the unit
    A[2, 0] = 0.99                                                                     # sets e = 0
    A[3, :] = -A[2, :]
    A[4, 5] = np.nextafter(1.0, 0.0) * 2.0 ** 30
    e = ozaki.row_exponents(A)
    X_ref = ozaki.fixed_point(A, e, S)
    X = ozaki.fixed_point_int(A, e, S)
    assert all(int(X[i, j]) == int(X_ref[i, j]) for i in range(A.shape[0]) for j in range(A.shape[1]))
    D_ref = ozaki.digits(X_ref, S)
    D = ozaki.digits_int(X, S)
    assert all(np.array_equal(a, b) for a, b in zip(D, D_ref))


def test_level9_largest_sum_closed_form():
    """Every value 127/128 is its own row maximum (e = 0) and has the fixed point 127 * 256^8: one
    leading digit 127, all others zero.  At level 9 the exact sum of an output is then
    K * 127^2 * 256^8 (the largest sum the emulated product can meet for a given K), and the
    result is K (127/128)^2 exactly."""
    K = 64
    A = np.full((2, K), 127.0 / 128.0)
    B = np.full((K, 3), -127.0 / 128.0)
    e, D = ozaki.slice_rows(A, 9)
    assert np.all(e == 0)
    assert np.all(D[0] == 127) and all(np.all(d == 0) for d in D[1:])
    C = ozaki.ozaki_gemm(A, B, 9, 9)
    assert np.all(C == -K * (127.0 / 128.0) ** 2)
    # the weight of the leading pair at level 9 is 256^(2*9 - 2) / 2^(2(8*9-1)) relative to 2^(ea+eb)
    Z = K * 127 * (-127) * 256 ** (2 * 9 - 2)
    assert ozaki.round_scaled(Z, -2 * (8 * 9 - 1)) == C[0, 0]
