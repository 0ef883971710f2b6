"""GPU parity of slicing, slice products and ozaki_gemm against the oracle (bit-exact)."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import ozaki

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_04795_gb300 as oz
    c = oz.Context(0)
    yield c
    c.close()


def _mat(rng, m, n, spread=True, zero_rows=(), special=False):
    A = rng.normal(size=(m, n))
    if spread:
        A *= 10.0 ** rng.uniform(-6, 0, size=(m, n))
    for r in zero_rows:
        if r < m:
            A[r] = 0.0
    if special and m > 3 and n > 3:
        A[1, 1] = 5e-310          # subnormal
        A[1, 2] = -3e-320
        A[2, :] = 1e-300          # tiny row
        A[3, 0] = 1e300           # huge
        A[3, 1] = -7e299
    return A


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("m,n,S", [(1, 1, 1), (5, 7, 2), (130, 70, 3), (257, 33, 7), (64, 300, 8), (9, 40, 9)])
def test_slice_bitexact(ctx, m, n, S):
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(m * 1000 + n + S)
    A = _mat(rng, m, n, zero_rows=(0,), special=True)
    dig, ex = oz.ozaki_slice(ctx, _dev(A), S)
    ctx.status()
    e_ref, D_ref = ozaki.slice_rows(A, S)
    assert np.array_equal(ex.cpu().numpy(), e_ref.astype(np.int32))
    for t in range(S):
        assert np.array_equal(dig[t].cpu().numpy().astype(np.int64), D_ref[t]), f"plane {t}"


@pytest.mark.parametrize("m,k,n,S", [(3, 5, 2, 2), (130, 70, 65, 3), (129, 300, 130, 4)])
def test_slice_products_exact_integers(ctx, m, k, n, S):
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(k)
    A, B = _mat(rng, m, k), _mat(rng, k, n)
    P = oz.ozaki_slice_products(ctx, _dev(A), _dev(B), S).cpu().numpy()
    ctx.status()
    _, DA = ozaki.slice_rows(A, S)
    _, DB = ozaki.slice_cols(B, S)
    for t in range(S):
        for u in range(S):
            ref = DA[t] @ DB[u]
            assert np.array_equal(P[t, u], ref.astype(np.float64)), (t, u)


CASES = [
    (1, 1, 1, 7, 7),
    (7, 9, 5, 3, 3),
    (129, 33, 65, 7, 7),      # ragged in every dimension, several tiles
    (130, 70, 130, 5, 9),     # level below the stored depth
    (64, 1100, 70, 7, 7),     # long K: mid-tile drains of the fuller diagonals
    (200, 260, 64, 8, 8),
    (33, 2050, 17, 2, 2),
    (40, 40, 40, 1, 1),
    (256, 64, 192, 4, 6),
    (7, 9, 5, 9, 9),          # level 9: two passes per tile (diagonals 0..7, then diagonal 8)
    (129, 33, 65, 9, 9),
    (64, 1100, 70, 9, 9),     # level 9, long K: staggered drains in the first pass, drains of
                              # diagonal 8 every 7 k-blocks in the second
]


@pytest.mark.parametrize("m,k,n,s,S", CASES)
def test_gemm_bitexact(ctx, m, k, n, s, S):
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(m + 7 * k + 13 * n + s)
    A = _mat(rng, m, k, zero_rows=(2,), special=(m > 4))
    B = _mat(rng, k, n)
    C = oz.ozaki_gemm(ctx, _dev(A), _dev(B), slices=S, level=s).cpu().numpy()
    ctx.status()
    ref = ozaki.ozaki_gemm(A, B, S, s)
    assert np.array_equal(C.view(np.int64), ref.view(np.int64)), np.argwhere(C != ref)[:5]


def test_gemm_alpha_beta(ctx):
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(11)
    A, B, C0 = _mat(rng, 70, 50), _mat(rng, 50, 90), rng.normal(size=(70, 90))
    Cd = _dev(C0)
    oz.ozaki_gemm(ctx, _dev(A), _dev(B), Cd, alpha=-0.5, beta=2.0, slices=6)
    ctx.status()
    ref = ozaki.ozaki_gemm(A, B, 6, alpha=-0.5, beta=2.0, C=C0)
    assert np.array_equal(Cd.cpu().numpy(), ref)


def test_gemm_strided_and_empty(ctx):
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(12)
    big = rng.normal(size=(40, 60))
    A = _dev(big)[:, :30]          # lda = 60 > k = 30
    B = _dev(rng.normal(size=(30, 20)))
    C = oz.ozaki_gemm(ctx, A, B, slices=7)
    ctx.status()
    assert np.array_equal(C.cpu().numpy(), ozaki.ozaki_gemm(big[:, :30], B.cpu().numpy(), 7))
    # k = 0: C = beta C
    C0 = torch.ones(4, 5, dtype=torch.float64, device="cuda")
    oz.ozaki_gemm(ctx, torch.zeros(4, 0, dtype=torch.float64, device="cuda"),
                  torch.zeros(0, 5, dtype=torch.float64, device="cuda"), C0, beta=3.0)
    ctx.status()
    assert torch.all(C0 == 3.0)
    # m = 0 is a no-op
    oz.ozaki_gemm(ctx, torch.zeros(0, 3, dtype=torch.float64, device="cuda"),
                  torch.zeros(3, 5, dtype=torch.float64, device="cuda"))
    ctx.status()


def test_gemm_rejects_bad_arguments(ctx):
    import paper_2510_04795_gb300 as oz
    A = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(oz.OzError) as ei:
        oz.ozaki_gemm(ctx, A, A, slices=10)
    assert ei.value.code == 1
    with pytest.raises(oz.OzError):
        oz.ozaki_gemm(ctx, A, A, slices=8, level=9)   # level above the stored depth


def test_gemm_level9_largest_sum_at_the_k_limit(ctx):
    """Level 9 at its longest reduction, K = 130,048, on the largest exact sum the 96-bit epilogue
    sums can meet: every value 127/128 (its own row maximum, leading digit 127), so each output is
    K * (127/128)^2 exactly, |Z| = K 127^2 2^64 just below 2^95.  One more column is refused at
    level 9 and accepted at level 8."""
    import paper_2510_04795_gb300 as oz
    k = 130048
    A = torch.full((3, k), 127.0 / 128.0, dtype=torch.float64, device="cuda")
    B = torch.full((k, 2), -127.0 / 128.0, dtype=torch.float64, device="cuda")
    C = oz.ozaki_gemm(ctx, A, B, slices=9, level=9)
    ctx.status()
    assert torch.all(C == -k * (127.0 / 128.0) ** 2)
    A1 = torch.full((3, k + 1), 127.0 / 128.0, dtype=torch.float64, device="cuda")
    B1 = torch.full((k + 1, 2), -127.0 / 128.0, dtype=torch.float64, device="cuda")
    with pytest.raises(oz.OzError):
        oz.ozaki_gemm(ctx, A1, B1, slices=9, level=9)
    C8 = oz.ozaki_gemm(ctx, A1, B1, slices=9, level=8)
    ctx.status()
    assert torch.all(C8 == -(k + 1) * (127.0 / 128.0) ** 2)


def test_nonfinite_input_reported(ctx):
    import paper_2510_04795_gb300 as oz
    A = torch.ones(8, 8, dtype=torch.float64, device="cuda")
    A[3, 4] = float("nan")
    oz.ozaki_gemm(ctx, A, A.clone().fill_(1.0))
    with pytest.raises(oz.OzError) as ei:
        ctx.status()
    assert ei.value.code == 2
    ctx.status()   # latch cleared


def test_native_mode_matches_fp64(ctx):
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(13)
    A, B = rng.normal(size=(100, 80)), rng.normal(size=(80, 60))
    C = oz.ozaki_gemm(ctx, _dev(A), _dev(B), mode="native").cpu().numpy()
    ctx.status()
    assert np.all(np.abs(C - A @ B) <= 1e-14 * (np.abs(A) @ np.abs(B)))


def test_gemm_error_within_bound_and_decreasing(ctx):
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(14)
    A, B = _mat(rng, 96, 300), _mat(rng, 300, 80)
    from fractions import Fraction
    ex = np.array([[float(sum(Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(300)))
                    for j in range(0, 80, 7)] for i in range(0, 96, 11)])
    prev = None
    for s in (2, 3, 4, 5, 6, 7, 8):
        C = oz.ozaki_gemm(ctx, _dev(A), _dev(B), slices=s).cpu().numpy()[::11, ::7]
        bnd = ozaki.error_bound(A, B, s)[::11, ::7]
        err = np.abs(C - ex)
        assert np.all(err <= bnd + np.spacing(np.abs(ex)) + np.spacing(np.abs(C)))
        mx = err.max()
        if prev is not None and prev > 1e-300:
            assert mx <= prev
        prev = mx


@pytest.mark.parametrize("scale_a,scale_b", [(1e-160, 1e-160), (1e-200, 1e-110), (1e150, 1e155), (2.0 ** -540, 2.0 ** -530)])
def test_gemm_extreme_exponents(ctx, scale_a, scale_b):
    """Results in the subnormal range, near overflow, and rounding across the normal/subnormal edge."""
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(15)
    A = rng.normal(size=(70, 40)) * scale_a
    B = rng.normal(size=(40, 65)) * scale_b
    A[0] *= 1e-6
    for S in (3, 7):
        C = oz.ozaki_gemm(ctx, _dev(A), _dev(B), slices=S).cpu().numpy()
        ctx.status()
        ref = ozaki.ozaki_gemm(A, B, S)
        assert np.array_equal(C.view(np.int64), ref.view(np.int64))


def test_performant_mode_dispatch(ctx):
    """Performant mode: each shape class is timed once both ways, the faster path runs, and the
    result is that path's, bit for bit; beta * C stays intact through the timing runs."""
    import paper_2510_04795_gb300 as oz
    g = torch.Generator(device="cuda").manual_seed(5)
    # tiny product: a cuBLAS DGEMM launch beats slicing plus the emulated GEMM
    A = torch.randn(32, 24, generator=g, device="cuda", dtype=torch.float64)
    B = torch.randn(24, 40, generator=g, device="cuda", dtype=torch.float64)
    C0 = torch.randn(32, 40, generator=g, device="cuda", dtype=torch.float64)
    assert oz.performant_choice(ctx, 32, 40, 24)[0] is None
    C = C0.clone()
    oz.ozaki_gemm(ctx, A, B, C, alpha=0.5, beta=2.0, mode="performant")
    mode, t_emu, t_nat = oz.performant_choice(ctx, 32, 40, 24)
    assert mode in ("eager", "native") and t_emu > 0 and t_nat > 0
    assert mode == ("eager" if t_emu <= t_nat else "native")
    ref = C0.clone()
    oz.ozaki_gemm(ctx, A, B, ref, alpha=0.5, beta=2.0, mode=mode)
    assert torch.equal(C, ref)
    # a second call of the same class (different sizes inside it) reuses the choice
    A2, B2 = A[:30, :20].contiguous(), B[:20, :33].contiguous()
    C2 = oz.ozaki_gemm(ctx, A2, B2, mode="performant")
    assert oz.performant_choice(ctx, 30, 33, 20)[1:] == (t_emu, t_nat)
    assert torch.equal(C2, oz.ozaki_gemm(ctx, A2, B2, mode=mode))
    # a large product: FP64 runs far below the emulated rate, so emulation is chosen
    A = torch.randn(4096, 4096, generator=g, device="cuda", dtype=torch.float64)
    B = torch.randn(4096, 4096, generator=g, device="cuda", dtype=torch.float64)
    C = oz.ozaki_gemm(ctx, A, B, mode="performant")
    mode, t_emu, t_nat = oz.performant_choice(ctx, 4096, 4096, 4096)
    assert mode == "eager" and t_emu < t_nat
    assert torch.equal(C, oz.ozaki_gemm(ctx, A, B, mode="eager"))
    ctx.status()
    # other entry points keep rejecting the mode
    st = synthetic.heff_structure(grid=(2, 2), dims=(2, 6), nterms=4, seed=1)
    blocks = [synthetic.gen_task_blocks(st, t, device="cuda") for t in range(st.ntask)]
    tasks = [(int(s), int(d), float(st.term_coef[k]), L, R) for (k, s, d), (L, R) in zip(st.tasks, blocks)]
    with pytest.raises(oz.OzError):
        oz.Heff(ctx, st.m, st.n, tasks, slices=7, mode="performant")
