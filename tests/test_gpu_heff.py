"""GPU parity of heff_apply against the oracle."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import heff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_04795_gb300 as oz
    c = oz.Context(0)
    yield c
    c.close()


def _problem(grid, dims, nterms, spread, seed=1, device="cuda"):
    st = synthetic.heff_structure(grid=grid, dims=dims, nterms=nterms, spread=spread, seed=seed)
    blocks = [synthetic.gen_task_blocks(st, t, device=device) for t in range(st.ntask)]
    psi = synthetic.gen_psi(st, device=device)
    return st, blocks, psi


def _tasks(st, blocks):
    return [(int(s), int(d), float(st.term_coef[k]), L, R) for (k, s, d), (L, R) in zip(st.tasks, blocks)]


@pytest.mark.parametrize("tile", ["cta", "pair"])
@pytest.mark.parametrize("seed,grid,dims,S,s", [(1, (3, 3), (2, 20), 7, 7), (2, (4, 3), (5, 70), 4, 4),
                                               (3, (3, 2), (60, 140), 9, 6), (4, (4, 4), (30, 300), 7, 7),
                                               (3, (3, 2), (60, 140), 9, 9)])
def test_heff_bitexact_vs_emulated_oracle(ctx, seed, grid, dims, S, s, tile):
    """Both tilings of the products (128 x 64 on one CTA; 256 x 64 on a CTA pair, with the pair's
    padding tile of odd operands and both stage-2 orientations) give the oracle's bits."""
    import paper_2510_04795_gb300 as oz
    st, blocks, psi = _problem(grid, dims, 8, True, seed)
    h = oz.Heff(ctx, st.m, st.n, _tasks(st, blocks), slices=S, level=s, tile=tile)
    assert h.info()["tile"] == (1 if tile == "cta" else 2)
    y = h.apply(psi)
    ctx.status()
    Lb = [b[0].cpu().numpy() for b in blocks]
    Rb = [b[1].cpu().numpy() for b in blocks]
    ref = heff.heff_apply_emulated(st, Lb, Rb, psi.cpu().numpy(), S, s)
    got = y.cpu().numpy()
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    h.close()


def test_heff_epilogue_layouts_bitexact(ctx):
    """Both epilogue layouts of the GEMM launches (16 owner warps; 8 owners with TMEM lane quarter 1
    handed over by a loader warp), in every combination over the two stages, give the oracle's bits;
    the automatic choice takes the hand-over layout for long tiles only."""
    import paper_2510_04795_gb300 as oz
    st, blocks, psi = _problem((4, 4), (30, 300), 8, True, 4)
    h = oz.Heff(ctx, st.m, st.n, _tasks(st, blocks), slices=7)
    Lb = [b[0].cpu().numpy() for b in blocks]
    Rb = [b[1].cpu().numpy() for b in blocks]
    ref = heff.heff_apply_emulated(st, Lb, Rb, psi.cpu().numpy(), 7)
    for e1 in (0, 1):
        for e2 in (0, 1):
            h.set_epilogue(e1, e2)
            inf = h.info()
            assert (inf["epilogue1"], inf["epilogue2"]) == (e1, e2)
            y = h.apply(psi)
            ctx.status()
            assert np.array_equal(y.cpu().numpy().view(np.int64), ref.view(np.int64)), (e1, e2)
    h.set_epilogue(-1, -1)
    with pytest.raises(oz.OzError):
        h.set_epilogue(2, 0)
    h.close()


def test_heff_repeatable_and_graph_replay(ctx):
    import paper_2510_04795_gb300 as oz
    st, blocks, psi = _problem((4, 4), (4, 60), 16, True, 5)
    h = oz.Heff(ctx, st.m, st.n, _tasks(st, blocks), slices=7)
    y1 = h.apply(psi).clone()
    y2 = h.apply(psi * 2.0)
    y3 = h.apply(psi)
    ctx.status()
    assert torch.equal(y1, y3)
    assert torch.equal(y2, 2.0 * y1)    # scaling psi by 2 scales every exponent exactly
    h.close()


def test_heff_40_blocks_slice_sweep(ctx):
    """40 sector blocks of 8..256, 128 terms, six-decade exponent spread: error vs FP64 per slice count."""
    import paper_2510_04795_gb300 as oz
    st, blocks, psi = _problem((8, 5), (8, 256), 128, True, 1)
    Lb = [b[0].cpu().numpy() for b in blocks]
    Rb = [b[1].cpu().numpy() for b in blocks]
    yref = heff.heff_apply_fp64(st, Lb, Rb, psi.cpu().numpy())
    errs = {}
    for s in (3, 4, 5, 6, 7, 8):
        h = oz.Heff(ctx, st.m, st.n, _tasks(st, blocks), slices=s)
        y = h.apply(psi)
        ctx.status()
        errs[s] = heff.rel_frobenius(y.cpu().numpy(), yref)
        h.close()
    print("rel Frobenius error by slice count:", errs)
    assert errs[7] <= 1e-12
    assert errs[8] <= 1e-13
    for a, b in zip((3, 4, 5), (4, 5, 6)):
        assert errs[b] < errs[a]


def test_heff_native_mode(ctx):
    import paper_2510_04795_gb300 as oz
    st, blocks, psi = _problem((5, 4), (8, 100), 32, True, 7)
    h = oz.Heff(ctx, st.m, st.n, _tasks(st, blocks), mode="native")
    y = h.apply(psi)
    ctx.status()
    Lb = [b[0].cpu().numpy() for b in blocks]
    Rb = [b[1].cpu().numpy() for b in blocks]
    yref = heff.heff_apply_fp64(st, Lb, Rb, psi.cpu().numpy())
    assert heff.rel_frobenius(y.cpu().numpy(), yref) < 1e-14
    h.close()


def test_heff_symmetric(ctx):
    import paper_2510_04795_gb300 as oz
    st, blocks, psi = _problem((4, 3), (4, 40), 16, False, 9)
    h = oz.Heff(ctx, st.m, st.n, _tasks(st, blocks), slices=7)
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn(h.dim, dtype=torch.float64, generator=g).cuda()
    z = torch.randn(h.dim, dtype=torch.float64, generator=g).cuda()
    hx, hz = h.apply(x).clone(), h.apply(z).clone()
    ctx.status()
    lhs, rhs = float(x @ hz), float(hx @ z)
    assert abs(lhs - rhs) <= 1e-13 * float(hx.norm() * z.norm())
    h.close()


def test_heff_per_sector_levels_bitexact(ctx):
    """The precision dial per block: random levels per stage-1 (source) and stage-2 (target)
    product reproduce the oracle's emulation with the same levels bit for bit; the carrier flops
    follow the levels; restoring the full level restores the default result."""
    import paper_2510_04795_gb300 as oz
    st, blocks, psi = _problem((4, 3), (5, 70), 8, True, 7)
    h = oz.Heff(ctx, st.m, st.n, _tasks(st, blocks), slices=7)
    y7 = h.apply(psi).clone()
    f7 = h.info()["carrier_flops"]
    rng = np.random.default_rng(3)
    s1 = [int(x) for x in rng.integers(3, 8, size=st.nsec)]
    s2 = [int(x) for x in rng.integers(3, 8, size=st.nsec)]
    h.set_levels(s1, s2)
    assert h.get_levels() == (s1, s2)
    y = h.apply(psi)
    ctx.status()
    Lb = [b[0].cpu().numpy() for b in blocks]
    Rb = [b[1].cpu().numpy() for b in blocks]
    ref = heff.heff_apply_emulated(st, Lb, Rb, psi.cpu().numpy(), 7, s1=s1, s2=s2)
    assert np.array_equal(y.cpu().numpy().view(np.int64), ref.view(np.int64))
    assert h.info()["carrier_flops"] < f7
    h.set_levels(None, None)
    assert torch.equal(h.apply(psi), y7)
    with pytest.raises(oz.OzError):
        h.set_levels([8] * st.nsec, None)      # above the handle's level
    h.close()


def test_heff_autotune_keeps_results(ctx):
    """The schedule autotuner times every tile schedule and keeps the fastest per stage; the
    product is bit-identical under every schedule."""
    import paper_2510_04795_gb300 as oz
    st, blocks, psi = _problem((5, 4), (8, 200), 24, False, 9)
    h = oz.Heff(ctx, st.m, st.n, _tasks(st, blocks), slices=7)
    y0 = h.apply(psi).clone()
    (s1, s2), ms = h.autotune(psi, reps=2)
    assert s1 in (0, 1, 2) and s2 in (0, 1, 2)
    assert len(ms) == 3 and all(a > 0 and b > 0 for a, b in ms)
    assert ms[s1][0] == min(m[0] for m in ms) and ms[s2][1] == min(m[1] for m in ms)
    assert torch.equal(h.apply(psi), y0)
    h.close()


@pytest.mark.parametrize("mode", ["eager", "native"])
def test_heff_update_ops_equals_fresh_handle(ctx, mode):
    """New operator values for the same structure: the product, the diagonal and (emulated) the
    captured graph's next replay equal those of a handle created from the new values."""
    import paper_2510_04795_gb300 as oz
    st, blocks, psi = _problem((4, 3), (5, 70), 16, True, 2)
    tasks_a = _tasks(st, blocks)
    blocks_b = [synthetic.gen_task_blocks(st, t, value_seed=9, device="cuda") for t in range(st.ntask)]
    tasks_b = [(s, d, 0.5 * c - 0.25, L, R) for (s, d, c, _, _), (L, R) in zip(tasks_a, blocks_b)]
    h = oz.Heff(ctx, st.m, st.n, tasks_a, slices=7, mode=mode)
    y_a = h.apply(psi).clone()
    h.update_ops(tasks_b)
    y_b = h.apply(psi)
    d_b = h.diag().clone()
    ctx.status()
    f = oz.Heff(ctx, st.m, st.n, tasks_b, slices=7, mode=mode)
    assert torch.equal(y_b, f.apply(psi))
    assert torch.equal(d_b, f.diag())
    assert not torch.equal(y_a, y_b)
    if mode == "eager":
        Lb = [b[0].cpu().numpy() for b in blocks_b]
        Rb = [b[1].cpu().numpy() for b in blocks_b]
        st_b = synthetic.HeffStructure(st.labels, st.m, st.n, st.term_delta, 0.5 * st.term_coef - 0.25, st.tasks,
                                       st.spread, st.seed)
        assert np.array_equal(y_b.cpu().numpy(), heff.heff_apply_emulated(st_b, Lb, Rb, psi.cpu().numpy(), 7))
    # errors: a different task count or sector pair is refused and leaves the handle usable
    with pytest.raises(oz.OzError):
        h.update_ops(tasks_b[:-1])
    s0, d0, c0, L0, R0 = tasks_b[0]
    bad = [(d0, s0, c0, L0, R0)] + tasks_b[1:] if s0 != d0 else None
    if bad is not None:
        with pytest.raises(oz.OzError):
            h.update_ops(bad)
    assert torch.equal(h.apply(psi), y_b)
    h.close()
    f.close()


def test_heff_update_ops_nonfinite(ctx):
    import paper_2510_04795_gb300 as oz
    st, blocks, psi = _problem((3, 3), (2, 20), 8, False, 1)
    tasks = _tasks(st, blocks)
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=5)
    y = h.apply(psi).clone()
    Lbad = tasks[0][3].clone()
    Lbad.view(-1)[0] = float("nan")
    with pytest.raises(oz.OzError):
        h.update_ops([(tasks[0][0], tasks[0][1], tasks[0][2], Lbad, tasks[0][4])] + tasks[1:])
    h.update_ops(tasks)
    assert torch.equal(h.apply(psi), y)
    h.close()
