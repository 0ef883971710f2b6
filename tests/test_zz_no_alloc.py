"""The allocation-free entry point (ozaki_gemm_noalloc) against the regular one (ozaki_gemm).

ozaki_gemm_noalloc serves callers that may not allocate device memory (for example code running
inside a host framework that owns the device memory pool, or inside a region that must not
synchronise the device).  It keeps its scratch in a fixed 64 MiB device array instead of a
workspace, so its results must be bit-identical to ozaki_gemm's; this file checks that on two
calls in a row (the second one reuses the array left over by the first), that later calls leave
the device's free memory unchanged, the k = 0 and reduced-level forms, and that a product whose
scratch would not fit is refused.  It is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _noalloc(lib, A, B, Cout, slices, level=0, alpha=1.0, beta=0.0):
    m, k = A.shape
    n = B.shape[1]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.ozaki_gemm_noalloc(m, n, k, float(alpha), A.data_ptr(), max(1, A.stride(0)), B.data_ptr(),
                                  max(1, B.stride(0)), float(beta), Cout.data_ptr(), Cout.stride(0), slices, level,
                                  stream)


def test_noalloc_matches_ozaki_gemm_twice():
    import paper_2510_04795_gb300 as oz
    from paper_2510_04795_gb300 import _native
    lib = _native.load()
    ctx = oz.Context(0)
    rng = np.random.default_rng(2024)
    cases = [(257, 300, 130, 7), (100, 64, 333, 5)]   # several tiles, ragged edges; second call differs
    for (m, k, n, S) in cases:
        A = torch.from_numpy(rng.normal(size=(m, k)) * 10.0 ** rng.uniform(-6, 0, size=(m, k))).cuda()
        B = torch.from_numpy(rng.normal(size=(k, n))).cuda()
        ref = oz.ozaki_gemm(ctx, A, B, slices=S)
        out = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
        rc = _noalloc(lib, A, B, out, S)
        torch.cuda.synchronize()
        ctx.status()
        assert rc == 0
        assert torch.equal(out.view(torch.int64), ref.view(torch.int64))
    ctx.close()


def test_noalloc_allocates_nothing_after_its_first_call():
    """Once the first call on the device has looked up the array, further calls (other shapes,
    other slice counts) change neither the device's free memory nor torch's allocator."""
    import paper_2510_04795_gb300 as oz
    from paper_2510_04795_gb300 import _native
    lib = _native.load()
    ctx = oz.Context(0)
    rng = np.random.default_rng(11)
    shapes = [(64, 40, 50, 7), (300, 200, 100, 7), (129, 17, 65, 4)]
    ops = []
    for (m, k, n, S) in shapes:
        A = torch.from_numpy(rng.normal(size=(m, k))).cuda()
        B = torch.from_numpy(rng.normal(size=(k, n))).cuda()
        ops.append((A, B, torch.empty((m, n), dtype=torch.float64, device="cuda"), S,
                    oz.ozaki_gemm(ctx, A, B, slices=S)))

    def rounds(n):
        for _ in range(n):
            for A, B, out, S, ref in ops:
                out.fill_(float("nan"))
                assert _noalloc(lib, A, B, out, S) == 0
                torch.cuda.synchronize()
                assert torch.equal(out.view(torch.int64), ref.view(torch.int64))

    # first round: the per-device set-up, and every kernel used below (the library's, and torch's
    # fill and compare) loaded once
    rounds(1)
    free0, _ = torch.cuda.mem_get_info()
    rounds(2)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # the calls alone take nothing from torch's allocator either
    n0 = torch.cuda.memory_stats()["allocation.all.allocated"]
    for A, B, out, S, _ in ops:
        assert _noalloc(lib, A, B, out, S) == 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_stats()["allocation.all.allocated"] == n0
    ctx.close()


def test_noalloc_alpha_beta_level_k0_and_limit():
    import paper_2510_04795_gb300 as oz
    from paper_2510_04795_gb300 import _native
    lib = _native.load()
    ctx = oz.Context(0)
    rng = np.random.default_rng(7)
    A = torch.from_numpy(rng.normal(size=(70, 50))).cuda()
    B = torch.from_numpy(rng.normal(size=(50, 90))).cuda()
    C0 = torch.from_numpy(rng.normal(size=(70, 90))).cuda()
    ref = oz.ozaki_gemm(ctx, A, B, C0.clone(), alpha=-0.5, beta=2.0, slices=6)
    out = C0.clone()
    assert _noalloc(lib, A, B, out, 6, alpha=-0.5, beta=2.0) == 0
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # a level below the slice count: the same kept pairs as ozaki_gemm at that level
    ref = oz.ozaki_gemm(ctx, A, B, slices=7, level=4)
    out = torch.empty_like(ref)
    assert _noalloc(lib, A, B, out, 7, level=4) == 0
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.int64), ref.view(torch.int64))
    # k = 0: C = beta C, as ozaki_gemm
    Ak = torch.empty((70, 0), dtype=torch.float64, device="cuda")
    Bk = torch.empty((0, 90), dtype=torch.float64, device="cuda")
    ref = oz.ozaki_gemm(ctx, Ak, Bk, C0.clone(), beta=-3.0, slices=7)
    out = C0.clone()
    assert _noalloc(lib, Ak, Bk, out, 7, beta=-3.0) == 0
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert torch.equal(out, -3.0 * C0)
    # 4096 x 4096 x 4096 at S = 7 needs far more than 64 MiB of scratch: refused, nothing launched
    big = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = lib.ozaki_gemm_noalloc(4096, 4096, 4096, 1.0, big.data_ptr(), 4096, big.data_ptr(), 4096, 0.0,
                                big.data_ptr(), 4096, 7, 0, C.c_void_p(0))
    assert rc == 1
    ctx.close()
