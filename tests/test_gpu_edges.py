"""Edge cases of the path on the GPU: sectors that receive no task, 1 x 1 blocks, zero and
non-finite psi, the host-buffer entry point, a one-dimensional eigenproblem, and sweeps of
degenerate systems (two orbitals, no electrons, a full shell)."""
import dataclasses

import numpy as np
import pytest
import torch

import synthetic
from oracle import dmrg as odmrg
from oracle import fci
from oracle import heff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_04795_gb300 as oz
    c = oz.Context(0)
    yield c
    c.close()


def _blocks(st):
    blocks = [synthetic.gen_task_blocks(st, t, device="cuda") for t in range(st.ntask)]
    tasks = [(int(s), int(d), float(st.term_coef[k]), L, R) for (k, s, d), (L, R) in zip(st.tasks, blocks)]
    return blocks, tasks


def _np(blocks):
    return [b[0].cpu().numpy() for b in blocks], [b[1].cpu().numpy() for b in blocks]


def test_sector_without_tasks_is_zero_and_bitexact(ctx):
    import paper_2510_04795_gb300 as oz
    st = synthetic.heff_structure(grid=(3, 3), dims=(3, 30), nterms=6, spread=True, seed=7)
    keep = np.array([d != 4 for (_, _, d) in st.tasks])            # nothing lands in sector 4
    st = dataclasses.replace(st, tasks=st.tasks[keep], partner=None)
    blocks, tasks = _blocks(st)
    psi = synthetic.gen_psi(st, device="cuda")
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=7)
    y = h.apply(psi)
    ctx.status()
    Lb, Rb = _np(blocks)
    ref = heff.heff_apply_emulated(st, Lb, Rb, psi.cpu().numpy(), 7)
    assert np.array_equal(y.cpu().numpy().view(np.int64), ref.view(np.int64))
    off = st.psi_offsets()
    assert not torch.any(y[off[4]:off[5]])
    h.close()


def test_one_by_one_blocks_bitexact(ctx):
    import paper_2510_04795_gb300 as oz
    st = synthetic.heff_structure(grid=(3, 2), dims=(1, 1), nterms=8, spread=True, seed=8)
    blocks, tasks = _blocks(st)
    psi = synthetic.gen_psi(st, device="cuda")
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=6)
    y = h.apply(psi)
    Lb, Rb = _np(blocks)
    ref = heff.heff_apply_emulated(st, Lb, Rb, psi.cpu().numpy(), 6)
    assert np.array_equal(y.cpu().numpy().view(np.int64), ref.view(np.int64))
    h.close()


def test_zero_and_nonfinite_psi(ctx):
    import paper_2510_04795_gb300 as oz
    from paper_2510_04795_gb300 import OzError
    st = synthetic.heff_structure(grid=(3, 3), dims=(3, 20), nterms=6, spread=False, seed=9)
    blocks, tasks = _blocks(st)
    psi = synthetic.gen_psi(st, device="cuda")
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=7)
    y0 = h.apply(psi).clone()
    assert not torch.any(h.apply(torch.zeros_like(psi)))
    bad = psi.clone()
    bad[5] = float("nan")
    h.apply(bad)
    with pytest.raises(OzError) as e:
        ctx.status()
    assert e.value.code == 2                                      # OZ_ENONFINITE, then cleared
    assert torch.equal(h.apply(psi), y0)
    ctx.status()
    h.close()


def test_host_entry_point_matches_device(ctx):
    import paper_2510_04795_gb300 as oz
    st = synthetic.heff_structure(grid=(4, 3), dims=(4, 40), nterms=8, spread=True, seed=10)
    blocks, tasks = _blocks(st)
    psi = synthetic.gen_psi(st, device="cuda")
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=7)
    y = h.apply(psi).cpu()
    yh = torch.empty_like(y).pin_memory()
    oz.heff_apply_host(h, psi.cpu().pin_memory(), yh)
    torch.cuda.synchronize()
    assert torch.equal(yh, y)
    h.close()


def test_davidson_one_dimensional(ctx):
    import paper_2510_04795_gb300 as oz
    L = torch.tensor([[3.0]], dtype=torch.float64, device="cuda")
    R = torch.tensor([[-0.5]], dtype=torch.float64, device="cuda")
    h = oz.Heff(ctx, [1], [1], [(0, 0, 2.0, L, R)], slices=7)
    x = torch.tensor([0.25], dtype=torch.float64, device="cuda")
    e, it, rc = oz.davidson_solve(h, x, tol=1e-12, max_iter=5)
    assert rc == 0 and it == 1 and e == -3.0 and abs(x.item()) == 1.0
    h.close()


@pytest.mark.parametrize("L,N,twosz", [(2, 2, 0), (3, 0, 0), (3, 6, 0), (3, 3, 1)])
def test_sweep_degenerate_systems(ctx, L, N, twosz):
    import paper_2510_04795_gb300 as oz
    h1, eri = synthetic.integrals(L, seed=4)
    got = oz.dmrg_sweep(ctx, h1, eri, N, twosz, 16, 1, slices=7)
    ref = np.array(odmrg.ExplicitDMRG(h1, eri, N, twosz, 16).sweep(1))
    assert np.max(np.abs(got - ref)) <= 1e-10
    if N == 0:
        assert np.all(got == 0.0)
    else:
        e_fci = fci.ground_state(h1, eri, N, twosz)[0]
        assert abs(got[-1] - e_fci) <= 1e-10
