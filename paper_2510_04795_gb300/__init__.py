"""GB300-native Ozaki-scheme emulated FP64 for the two-site DMRG effective-Hamiltonian product.

Thin Python binding over the C ABI of libozdmrg (include/ozdmrg.h); torch supplies device
memory and streams only.  Names follow the C ABI: ``ozaki_gemm``, ``ozaki_slice``,
``ozaki_slice_products``, ``heff_apply`` (on an ``Heff`` handle), ``davidson_step`` (on a
``Davidson`` state), ``davidson_solve``, ``symeig_small``, ``dmrg_sweep`` (and the ``DMRG`` handle), the
per-block precision dial (``Heff.set_levels``, ``Heff.select_levels``) and the selector network ``MLP``.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N
from ._native import OzError, OZ_MODE_EAGER, OZ_MODE_NATIVE, OZ_NFEAT

SELECTORS = {"fixed": N.OZ_SELECT_FIXED, "analytic": N.OZ_SELECT_ANALYTIC, "learned": N.OZ_SELECT_LEARNED}

__all__ = ["Context", "Heff", "Davidson", "OzError", "ozaki_gemm", "performant_choice", "ozaki_slice", "ozaki_slice_products",
           "heff_apply", "heff_apply_host", "heff_stage_times", "heff_ops_times", "davidson_solve", "symeig_small", "DMRG",
           "dmrg_sweep", "MLP", "OZ_NFEAT", "SELECTORS", "lanczos_solve", "heff_partition", "reduce_ordered",
           "ShardedHeff",
           "OZ_MODE_EAGER", "OZ_MODE_NATIVE"]


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _prec(slices: int, level: int, mode, tile="auto") -> N.oz_prec:
    m = {"eager": OZ_MODE_EAGER, "native": OZ_MODE_NATIVE, "performant": N.OZ_MODE_PERFORMANT}.get(mode, mode)
    t = {"auto": N.OZ_TILE_AUTO, "cta": N.OZ_TILE_CTA, "pair": N.OZ_TILE_PAIR}.get(tile, tile)
    return N.oz_prec(int(slices), int(level), int(m), int(t))


def _check_f64(*ts):
    for t in ts:
        if t.dtype != torch.float64 or not t.is_cuda:
            raise OzError(N.OZ_EINVAL, "expected a CUDA float64 tensor")


class Context:
    """One libozdmrg context (device workspace + error latch) on a CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = N.load()
        self.device = device
        h = C.c_void_p()
        N.check(self.lib.oz_ctx_create(C.byref(h), device))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.oz_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None):
        """Synchronise and raise OzError if a device-side fault was latched."""
        N.check(self.lib.oz_status(self.h, _stream(stream)))


def ozaki_gemm(ctx: Context, A: torch.Tensor, B: torch.Tensor, C_out: torch.Tensor | None = None, alpha=1.0,
               beta=0.0, slices=7, level=0, mode="eager", stream=None) -> torch.Tensor:
    """C = alpha * (A B) + beta * C, emulated FP64 (row-major CUDA float64 tensors)."""
    _check_f64(A, B)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise OzError(N.OZ_EINVAL, "inner dimensions differ")
    if A.stride(1) != 1 or B.stride(1) != 1:
        raise OzError(N.OZ_EINVAL, "A and B need unit column stride")
    if C_out is None:
        C_out = torch.zeros(m, n, dtype=torch.float64, device=A.device)
    _check_f64(C_out)
    p = _prec(slices, level, mode)
    N.check(ctx.lib.ozaki_gemm(ctx.h, m, n, k, float(alpha), _ptr(A), max(A.stride(0), 1), _ptr(B),
                               max(B.stride(0), 1), float(beta), _ptr(C_out), max(C_out.stride(0), 1),
                               C.byref(p), _stream(stream)))
    return C_out


def performant_choice(ctx: Context, m: int, n: int, k: int, slices=7, level=0):
    """(mode, emulated ms, native ms) that ``mode="performant"`` chose for the shape class of
    (m, n, k); mode is "eager", "native" or None when no call of that class has run yet."""
    p = _prec(slices, level, "eager")
    md = C.c_int()
    ms = (C.c_float * 2)()
    N.check(ctx.lib.oz_performant_choice(ctx.h, int(m), int(n), int(k), C.byref(p), C.byref(md), ms))
    name = {OZ_MODE_EAGER: "eager", OZ_MODE_NATIVE: "native"}.get(md.value)
    return name, ms[0], ms[1]


def ozaki_slice(ctx: Context, A: torch.Tensor, slices: int, stream=None):
    """(digits int8 [S, rows, cols], exponents int32 [rows]) of the rows of A."""
    _check_f64(A)
    rows, cols = A.shape
    dig = torch.empty(slices, rows, cols, dtype=torch.int8, device=A.device)
    ex = torch.empty(rows, dtype=torch.int32, device=A.device)
    N.check(ctx.lib.ozaki_slice(ctx.h, rows, cols, _ptr(A), A.stride(0), slices, _ptr(dig), _ptr(ex),
                                _stream(stream)))
    return dig, ex


def ozaki_slice_products(ctx: Context, A: torch.Tensor, B: torch.Tensor, slices: int, stream=None):
    """Every slice product P[t, u] = A^t B^u as exact integers in float64, shape [S, S, m, n]."""
    _check_f64(A, B)
    m, k = A.shape
    n = B.shape[1]
    P = torch.empty(slices, slices, m, n, dtype=torch.float64, device=A.device)
    N.check(ctx.lib.ozaki_slice_products(ctx.h, m, n, k, _ptr(A), A.stride(0), _ptr(B), B.stride(0), slices,
                                         _ptr(P), _stream(stream)))
    return P


def _task_array(tasks):
    arr = (N.oz_task * max(1, len(tasks)))()
    for i, (s, d, c, L, R) in enumerate(tasks):
        _check_f64(L, R)
        if not (L.is_contiguous() and R.is_contiguous()):
            raise OzError(N.OZ_EINVAL, "task blocks must be contiguous")
        arr[i] = N.oz_task(int(s), int(d), float(c), _ptr(L), _ptr(R))
    return arr


class Heff:
    """Block-sparse two-site H_eff handle: Y = sum over tasks of coef * L psi[src] R^T into Y[dst].

    ``tasks`` is a sequence of (src, dst, coef, L, R) with L (m[dst] x m[src]) and
    R (n[dst] x n[src]) CUDA float64 tensors (kept alive by the handle in native mode).
    """

    def __init__(self, ctx: Context, m, n, tasks, slices=7, level=0, mode="eager", tile="auto"):
        """``tile``: "cta" (128 x 64 tiles, one CTA each), "pair" (256 x 64 tiles on CTA pairs) or
        "auto" (= "cta", the faster on GB300); the results are identical."""
        self.ctx = ctx
        self.lib = ctx.lib
        self.m = [int(x) for x in m]
        self.n = [int(x) for x in n]
        nsec = len(self.m)
        arr = _task_array(tasks)
        mm = (C.c_int * nsec)(*self.m)
        nn = (C.c_int * nsec)(*self.n)
        p = _prec(slices, level, mode, tile)
        h = C.c_void_p()
        N.check(self.lib.oz_heff_create(ctx.h, nsec, mm, nn, len(tasks), arr, C.byref(p), C.byref(h)))
        self.h = h
        self.dim = sum(a * b for a, b in zip(self.m, self.n))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.oz_heff_destroy(self.h)
            self.h = C.c_void_p()

    def update_ops(self, tasks):
        """New coef, L and R for the same (src, dst) task list; the next product equals that of a
        handle created from ``tasks`` (allocations, schedules, levels and graph are kept)."""
        N.check(self.lib.oz_heff_update_ops(self.h, len(tasks), _task_array(tasks)))

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def set_epilogue(self, e1: int = -1, e2: int = -1):
        """Epilogue layout of the stage-1 / stage-2 GEMM launches (0, 1, -1 = automatic); the results
        are identical (``oz_heff_set_epilogue``)."""
        N.check(self.lib.oz_heff_set_epilogue(self.h, int(e1), int(e2)))

    def info(self) -> dict:
        inf = N.oz_heff_info()
        N.check(self.lib.oz_heff_info_get(self.h, C.byref(inf)))
        return {f: getattr(inf, f) for f, _ in N.oz_heff_info._fields_}

    def apply(self, psi: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        _check_f64(psi)
        if y is None:
            y = torch.empty_like(psi)
        N.check(self.lib.heff_apply(self.h, _ptr(psi), _ptr(y), _stream(stream)))
        return y

    def set_levels(self, s1=None, s2=None):
        """Per-sector slice levels: s1[q] for the stage-1 product of source sector q, s2[q] for the
        stage-2 product of target sector q (None = the handle's level)."""
        nsec = len(self.m)
        a = (C.c_int * nsec)(*[int(x) for x in s1]) if s1 is not None else None
        b = (C.c_int * nsec)(*[int(x) for x in s2]) if s2 is not None else None
        N.check(self.lib.oz_heff_set_levels(self.h, a, b))

    def autotune(self, psi: torch.Tensor, reps: int = 2, stream=None):
        """Time every tile schedule of the two stages and keep the fastest: ((sched1, sched2),
        [(stage-1 ms, stage-2 ms) per schedule])."""
        _check_f64(psi)
        sc = (C.c_int * 2)()
        ms = (C.c_float * 6)()
        N.check(self.lib.oz_heff_autotune(self.h, _ptr(psi), int(reps), sc, ms, _stream(stream)))
        return (sc[0], sc[1]), [(ms[2 * c], ms[2 * c + 1]) for c in range(3)]

    def get_levels(self):
        nsec = len(self.m)
        a, b = (C.c_int * nsec)(), (C.c_int * nsec)()
        N.check(self.lib.oz_heff_get_levels(self.h, a, b))
        return list(a), list(b)

    def problem_features(self, psi: torch.Tensor, stream=None):
        """(feat1, feat2): nsec x OZ_NFEAT float32 numpy arrays of the stage-1 / stage-2 products."""
        import numpy as np
        _check_f64(psi)
        nsec = len(self.m)
        f1 = np.zeros((nsec, OZ_NFEAT), dtype=np.float32)
        f2 = np.zeros((nsec, OZ_NFEAT), dtype=np.float32)
        N.check(self.lib.oz_heff_problem_features(self.h, _ptr(psi), f1.ctypes.data, f2.ctypes.data,
                                                  _stream(stream)))
        return f1, f2

    def problem_errors(self, psi: torch.Tensor, level: int, stream=None):
        """(err1, err2): relative errors of every product at `level` against the handle's level."""
        import numpy as np
        _check_f64(psi)
        nsec = len(self.m)
        e1, e2 = np.zeros(nsec), np.zeros(nsec)
        N.check(self.lib.oz_heff_problem_errors(self.h, _ptr(psi), int(level), e1.ctypes.data, e2.ctypes.data,
                                                _stream(stream)))
        return e1, e2

    def select_levels(self, psi: torch.Tensor, selector="learned", budget=1e-12, net=None, margin=0.5,
                      stream=None):
        """Pick and set per-product levels (see oz_heff_select_levels); returns (s1, s2)."""
        _check_f64(psi)
        nsec = len(self.m)
        a, b = (C.c_int * nsec)(), (C.c_int * nsec)()
        sel = SELECTORS.get(selector, selector)
        N.check(self.lib.oz_heff_select_levels(self.h, _ptr(psi), int(sel), float(budget),
                                               net.h if net is not None else None, float(margin), a, b,
                                               _stream(stream)))
        return list(a), list(b)

    def diag(self, stream=None) -> torch.Tensor:
        """Diagonal of H_eff (the Davidson preconditioner), length dim."""
        out = torch.empty(self.dim, dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        N.check(self.lib.oz_heff_diag(self.h, _ptr(out), _stream(stream)))
        return out


class Davidson:
    """Davidson state for the lowest eigenpair of an ``Heff`` (all vector work on the device)."""

    def __init__(self, heff: Heff, max_sub: int = 24, tol: float = 1e-10):
        self.heff = heff
        self.lib = heff.lib
        h = C.c_void_p()
        N.check(self.lib.oz_davidson_create(heff.h, int(max_sub), float(tol), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.oz_davidson_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def start(self, x0: torch.Tensor, stream=None):
        _check_f64(x0)
        N.check(self.lib.davidson_start(self.h, _ptr(x0), _stream(stream)))

    def step(self, stream=None):
        """One iteration: (theta, |r|, converged).  Raises OzError(OZ_ENOCONV) on breakdown."""
        th, rs, cv = C.c_double(), C.c_double(), C.c_int()
        N.check(self.lib.davidson_step(self.h, C.byref(th), C.byref(rs), C.byref(cv), _stream(stream)))
        return th.value, rs.value, bool(cv.value)

    def ritz(self, stream=None) -> torch.Tensor:
        x = torch.empty(self.heff.dim, dtype=torch.float64, device=f"cuda:{self.heff.ctx.device}")
        N.check(self.lib.davidson_ritz(self.h, _ptr(x), _stream(stream)))
        return x


def heff_apply_host(h: Heff, psi_host: torch.Tensor, y_host: torch.Tensor, stream=None) -> torch.Tensor:
    """End-to-end product on host (preferably pinned) float64 tensors."""
    if psi_host.is_cuda or y_host.is_cuda or psi_host.dtype != torch.float64 or y_host.dtype != torch.float64:
        raise OzError(N.OZ_EINVAL, "expected host float64 tensors")
    N.check(h.lib.heff_apply_host(h.h, psi_host.data_ptr(), y_host.data_ptr(), _stream(stream)))
    return y_host


def heff_partition(m, n, src, dst, world: int):
    """Owner rank of every task (host computation, no GPU): a balanced, deterministic split of the
    task list over ``world`` ranks by FP64 flop cost (``oz_heff_partition``)."""
    import numpy as np
    lib = N.load()
    m = np.ascontiguousarray(m, dtype=np.int32)
    n = np.ascontiguousarray(n, dtype=np.int32)
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    owner = np.zeros(len(src), dtype=np.int32)
    N.check(lib.oz_heff_partition(len(m), m.ctypes.data, n.ctypes.data, len(src), src.ctypes.data,
                                  dst.ctypes.data, int(world), owner.ctypes.data))
    return owner


def reduce_ordered(parts, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """out = ((parts[0] + parts[1]) + parts[2]) + ... elementwise in FP64 (CUDA tensors, one
    rounding per addition in list order)."""
    _check_f64(*parts)
    if out is None:
        out = torch.empty_like(parts[0])
    arr = (C.c_void_p * len(parts))(*[p.data_ptr() for p in parts])
    N.check(N.load().oz_reduce_ordered(arr, len(parts), parts[0].numel(), _ptr(out), _stream(stream)))
    return out


def heff_apply_streamed(ctx: Context, m, n, tasks, psi: torch.Tensor, chunks: int, y: torch.Tensor | None = None,
                        slices=7, level=0, mode="eager", stream=None) -> torch.Tensor:
    """H_eff psi for structures whose operator digits do not fit on the device at once
    (``oz_heff_apply_streamed``): the tasks split into ``chunks`` groups as ``heff_partition`` splits
    them over ranks, each group's handle built, applied and released in turn, the partial products
    summed in group order -- the term-sharded product over ``chunks`` ranks, on one GPU."""
    _check_f64(psi)
    m = [int(x) for x in m]
    n = [int(x) for x in n]
    if y is None:
        y = torch.empty_like(psi)
    _check_f64(y)
    nsec = len(m)
    p = _prec(slices, level, mode)
    N.check(ctx.lib.oz_heff_apply_streamed(ctx.h, nsec, (C.c_int * nsec)(*m), (C.c_int * nsec)(*n), len(tasks),
                                           _task_array(tasks), C.byref(p), int(chunks), _ptr(psi), _ptr(y),
                                           _stream(stream)))
    return y


class ShardedHeff:
    """This rank's share of a term-sharded H_eff: a handle built from the tasks that
    ``heff_partition`` gives to ``rank``; ``apply`` computes the partial product, gathers the
    partial vectors of all ranks over ``torch.distributed`` (``group``) and sums them in rank
    order with ``reduce_ordered``.  With world = 1 it is the unsharded product."""

    def __init__(self, ctx: Context, m, n, tasks, rank: int, world: int, group=None, slices=7, level=0,
                 mode="eager"):
        owner = heff_partition(m, n, [t[0] for t in tasks], [t[1] for t in tasks], world)
        self.rank, self.world, self.group = int(rank), int(world), group
        self.owned = [i for i, o in enumerate(owner) if o == rank]
        self.local = Heff(ctx, m, n, [tasks[i] for i in self.owned], slices=slices, level=level, mode=mode)
        self.dim = self.local.dim

    def apply_partial(self, psi: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
        return self.local.apply(psi, y)

    def apply(self, psi: torch.Tensor) -> torch.Tensor:
        part = self.local.apply(psi)
        if self.world == 1:
            return part
        import torch.distributed as dist
        parts = [torch.empty_like(part) for _ in range(self.world)]
        dist.all_gather(parts, part, group=self.group)
        return reduce_ordered(parts)

    def close(self):
        self.local.close()


def heff_ops_times(h: Heff):
    """([rowmax ms, digits ms], [rowmax bytes, digits bytes]) of the handle's last operator slicing."""
    ms = (C.c_float * 2)()
    by = (C.c_longlong * 2)()
    N.check(h.lib.oz_heff_ops_times(h.h, ms, by))
    return [float(x) for x in ms], [int(x) for x in by]


def heff_stage_times(h: Heff) -> list:
    """Device ms of [psi slicing, stage-1 GEMM, intermediate slicing, stage-2 GEMM] of the last product."""
    arr = (C.c_float * 4)()
    N.check(h.lib.oz_heff_stage_times(h.h, arr))
    return [float(x) for x in arr]


def heff_apply(h: Heff, psi: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    return h.apply(psi, y, stream)


def davidson_solve(h: Heff, psi: torch.Tensor, tol: float = 1e-10, max_iter: int = 200, stream=None):
    """Lowest eigenpair of H_eff from the start vector psi (overwritten with the Ritz vector).

    Returns (energy, iterations, status) with status OZ_OK or OZ_ENOCONV; other errors raise."""
    _check_f64(psi)
    e, it = C.c_double(), C.c_int()
    rc = h.lib.davidson_solve(h.h, _ptr(psi), float(tol), int(max_iter), C.byref(e), C.byref(it), _stream(stream))
    if rc not in (N.OZ_OK, N.OZ_ENOCONV):
        N.check(rc)
    return e.value, it.value, rc


def lanczos_solve(h: Heff, psi: torch.Tensor, eps: float = 1e-10, max_iter: int = 500, krylov: int = 30,
                  stream=None):
    """Lowest eigenpair by Lanczos (full reorthogonalisation, explicit restart): (energy,
    products, status) with status OZ_OK or OZ_ENOCONV; psi is overwritten by the Ritz vector."""
    _check_f64(psi)
    e, it = C.c_double(), C.c_int()
    rc = h.lib.lanczos_solve(h.h, _ptr(psi), float(eps), int(max_iter), int(krylov), C.byref(e), C.byref(it),
                             _stream(stream))
    if rc not in (N.OZ_OK, N.OZ_ENOCONV):
        N.check(rc)
    return e.value, it.value, rc


def symeig_small(G: torch.Tensor, stream=None):
    """(eigenvalues ascending, eigenvectors as columns) of a symmetric m x m CUDA float64 matrix, m <= 32."""
    _check_f64(G)
    m = G.shape[0]
    w = torch.empty(m, dtype=torch.float64, device=G.device)
    V = torch.empty(m, m, dtype=torch.float64, device=G.device)
    N.check(N.load().oz_symeig_small(_ptr(G), m, G.stride(0), _ptr(w), _ptr(V), m, _stream(stream)))
    return w, V


def _host_integrals(h1, eri):
    import numpy as np
    h1 = np.ascontiguousarray(np.asarray(h1, dtype=np.float64))
    eri = np.ascontiguousarray(np.asarray(eri, dtype=np.float64))
    L = h1.shape[0]
    if h1.shape != (L, L) or eri.size != L ** 4:
        raise OzError(N.OZ_EINVAL, "h1 must be L x L and eri L^4")
    return h1, eri, L


class DMRG:
    """Two-site DMRG of the ab initio Hamiltonian (h1, eri host arrays, chemist notation)."""

    def __init__(self, ctx: Context, h1, eri, nelec: int, twosz: int, D: int, slices=7, level=0, mode="eager",
                 tol: float = 1e-10, seed: int = 0):
        self.ctx = ctx
        self.lib = ctx.lib
        self._h1, self._eri, self.L = _host_integrals(h1, eri)
        p = _prec(slices, level, mode)
        h = C.c_void_p()
        N.check(self.lib.oz_dmrg_create(ctx.h, self._h1.ctypes.data, self._eri.ctypes.data, self.L, int(nelec),
                                        int(twosz), int(D), C.byref(p), float(tol), int(seed), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.oz_dmrg_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def set_prediction(self, on: bool = True):
        """Start each bond's eigensolver from the previous bond's transformed solution (default)."""
        N.check(self.lib.oz_dmrg_set_prediction(self.h, 1 if on else 0))

    def set_solver(self, solver="davidson", tol=1e-10, check_fp64=False):
        """Eigensolver of the two-site update ("davidson" or "lanczos") and its tolerance;
        check_fp64 re-evaluates every Ritz vector with the FP64 H_eff and flags non-variational
        Ritz values in steps()."""
        code = {"davidson": 0, "lanczos": 1}[solver]
        N.check(self.lib.oz_dmrg_set_solver(self.h, code, float(tol), int(bool(check_fp64))))

    def set_rdm(self, slices=7, level=0, mode="eager"):
        """Precision of the density matrices of the truncation (default: native FP64)."""
        p = _prec(slices, level, mode)
        N.check(self.lib.oz_dmrg_set_rdm_prec(self.h, C.byref(p)))

    def set_renorm(self, slices=7, level=0, mode="eager"):
        """Precision of the renormalisation products U^T O U (default: native FP64)."""
        p = _prec(slices, level, mode)
        N.check(self.lib.oz_dmrg_set_renorm_prec(self.h, C.byref(p)))

    def run(self, nsweeps: int):
        """Runs nsweeps sweeps; returns the 2 (L - 1) nsweeps bond energies."""
        import numpy as np
        e = np.zeros(max(1, 2 * (self.L - 1) * nsweeps))
        N.check(self.lib.oz_dmrg_run(self.h, int(nsweeps), e.ctypes.data))
        return e[: 2 * (self.L - 1) * nsweeps]

    def steps(self) -> list:
        n = C.c_int()
        N.check(self.lib.oz_dmrg_steps(self.h, None, 0, C.byref(n)))
        arr = (N.oz_dmrg_step * max(1, n.value))()
        N.check(self.lib.oz_dmrg_steps(self.h, arr, n.value, C.byref(n)))
        return [{f: getattr(arr[i], f) for f, _ in N.oz_dmrg_step._fields_} for i in range(n.value)]

    def set_trace(self, stride: int):
        """Record every stride-th emulated renormalisation / density-matrix product from now on
        (0 = off; clears the record)."""
        N.check(self.lib.oz_dmrg_set_trace(self.h, int(stride)))

    def trace(self) -> list:
        """The recorded products: dicts with kind (0: T = O U, 1: U^T T, 2: density matrix), step,
        slices, level and the host arrays A (op(A)), B (op(B)) and C (the emulated result)."""
        import numpy as np
        n = C.c_longlong()
        N.check(self.lib.oz_dmrg_trace(self.h, -1, None, None, None, None, C.byref(n)))
        out = []
        info = (C.c_int * 7)()
        for i in range(n.value):
            N.check(self.lib.oz_dmrg_trace(self.h, i, info, None, None, None, None))
            kind, step, m, nn, k, S, lv = list(info)
            A, B, Cm = np.empty((m, k)), np.empty((k, nn)), np.empty((m, nn))
            N.check(self.lib.oz_dmrg_trace(self.h, i, None, A.ctypes.data, B.ctypes.data, Cm.ctypes.data, None))
            out.append({"kind": kind, "step": step, "slices": S, "level": lv, "A": A, "B": B, "C": Cm})
        return out

    def bond_heff(self, bond: int, psi: torch.Tensor | None = None, stream=None):
        """(H_eff psi or None, determinant pattern of every two-site basis state) at a bond."""
        import numpy as np
        dim = C.c_longlong()
        N.check(self.lib.oz_dmrg_bond_heff(self.h, int(bond), None, None, None, C.byref(dim), _stream(stream)))
        pats = np.zeros(dim.value, dtype=np.int64)
        y = None
        if psi is not None:
            _check_f64(psi)
            if psi.numel() != dim.value:
                raise OzError(N.OZ_EINVAL, "psi has the wrong length")
            y = torch.empty_like(psi)
        N.check(self.lib.oz_dmrg_bond_heff(self.h, int(bond), _ptr(psi) if psi is not None else None,
                                           _ptr(y) if y is not None else None, pats.ctypes.data, C.byref(dim),
                                           _stream(stream)))
        return y, pats


def dmrg_sweep(ctx: Context, h1, eri, nelec: int, twosz: int, D: int, nsweeps: int, slices=7, level=0,
               mode="eager", tol: float = 1e-10, seed: int = 0):
    """One-shot sweep run; returns the 2 (L - 1) nsweeps bond energies."""
    import numpy as np
    h1, eri, L = _host_integrals(h1, eri)
    p = _prec(slices, level, mode)
    e = np.zeros(max(1, 2 * (L - 1) * nsweeps))
    N.check(ctx.lib.dmrg_sweep(ctx.h, h1.ctypes.data, eri.ctypes.data, L, int(nelec), int(twosz), int(D),
                               int(nsweeps), C.byref(p), float(tol), int(seed), e.ctypes.data))
    return e[: 2 * (L - 1) * nsweeps]


class MLP:
    """Selector network (two tanh hidden layers, FP32) trained on the device by its own kernels."""

    def __init__(self, nin: int = OZ_NFEAT, nhidden: int = 64, nout: int = 6, seed: int = 4):
        self.lib = N.load()
        h = C.c_void_p()
        N.check(self.lib.oz_mlp_create(int(nin), int(nhidden), int(nout), int(seed), C.byref(h)))
        self.h = h
        self.nin, self.nhidden, self.nout = nin, nhidden, nout

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.oz_mlp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        import numpy as np
        out = np.zeros(self.lib.oz_mlp_param_count(self.h), dtype=np.float32)
        N.check(self.lib.oz_mlp_get_params(self.h, out.ctypes.data))
        return out

    def set_params(self, flat):
        import numpy as np
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        N.check(self.lib.oz_mlp_set_params(self.h, flat.ctypes.data))

    def forward(self, X: torch.Tensor, stream=None) -> torch.Tensor:
        X = X.contiguous()
        Y = torch.empty(X.shape[0], self.nout, dtype=torch.float32, device=X.device)
        N.check(self.lib.oz_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(Y), _stream(stream)))
        return Y

    def gradient(self, X, T, M, stream=None):
        """(loss, flat gradient) over all rows."""
        import numpy as np
        g = np.zeros(self.lib.oz_mlp_param_count(self.h), dtype=np.float32)
        loss = C.c_float()
        N.check(self.lib.oz_mlp_gradient(self.h, _ptr(X), _ptr(T), _ptr(M), X.shape[0], C.byref(loss), g.ctypes.data,
                                         _stream(stream)))
        return loss.value, g

    def train(self, X, T, M, epochs=200, batch=64, lr=1e-3, seed=5, stream=None) -> float:
        loss = C.c_float()
        N.check(self.lib.oz_mlp_train(self.h, _ptr(X), _ptr(T), _ptr(M), X.shape[0], int(epochs), int(batch),
                                      float(lr), int(seed), C.byref(loss), _stream(stream)))
        return loss.value
