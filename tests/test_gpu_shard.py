"""Term-sharded H_eff psi on one GPU: the handles of every rank of a world-2 (and world-3) split,
built in one process, each partial product bit-exact against the oracle's emulated product of
that rank's tasks, and their rank-ordered sum (oz_reduce_ordered) against the unsharded product.
No rank waits on another here: the partial products run one after the other."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import heff

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_partials_and_ordered_sum(world):
    import paper_2510_04795_gb300 as oz
    ctx = oz.Context(0)
    st = synthetic.heff_structure(grid=(4, 4), dims=(8, 96), nterms=16, spread=True, seed=7)
    blocks = [tuple(b.cuda() for b in synthetic.gen_task_blocks(st, t)) for t in range(st.ntask)]
    psi = synthetic.gen_psi(st).cuda()
    tasks = [(int(s), int(d), float(st.term_coef[k]), L, R) for (k, s, d), (L, R) in zip(st.tasks, blocks)]
    Lb = [b[0].cpu().numpy() for b in blocks]
    Rb = [b[1].cpu().numpy() for b in blocks]
    psi_h = psi.cpu().numpy()
    full = oz.Heff(ctx, st.m, st.n, tasks, slices=7)
    y_full = full.apply(psi)
    parts = []
    for rank in range(world):
        sh = oz.ShardedHeff(ctx, st.m, st.n, tasks, rank, world, slices=7)
        p = sh.apply_partial(psi)
        ids = np.array(sh.owned, dtype=np.int64)
        sub = synthetic.HeffStructure(st.labels, st.m, st.n, st.term_delta, st.term_coef, st.tasks[ids], st.spread,
                                      st.seed)
        ref = heff.heff_apply_emulated(sub, [Lb[i] for i in ids], [Rb[i] for i in ids], psi_h, 7)
        assert np.array_equal(p.cpu().numpy().view(np.int64), ref.view(np.int64)), rank
        parts.append(p)
        sh.close()
    y = oz.reduce_ordered(parts)
    ctx.status()
    # the reduction is the rank-ordered FP64 sum, bit for bit
    acc = parts[0].cpu().numpy().copy()
    for p in parts[1:]:
        acc = acc + p.cpu().numpy()
    assert np.array_equal(y.cpu().numpy(), acc)
    ref64 = heff.heff_apply_fp64(st, Lb, Rb, psi_h)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(y.cpu().numpy(), y_full.cpu().numpy()) <= 1e-13
    assert rel(y.cpu().numpy(), ref64) <= 1e-12
    full.close()
    ctx.close()


def test_reduce_ordered_edge_cases():
    import paper_2510_04795_gb300 as oz
    from paper_2510_04795_gb300 import OzError
    x = torch.arange(1000, dtype=torch.float64, device="cuda") * 0.1
    y = oz.reduce_ordered([x])                      # one part: a copy
    assert torch.equal(x, y)
    out = x.clone()
    oz.reduce_ordered([out, x, x], out=out)         # out may alias the first part
    assert torch.equal(out, (x + x) + x)
    with pytest.raises(OzError):
        oz.reduce_ordered([x] * 65)


@pytest.mark.parametrize("chunks", [1, 3])
def test_streamed_product_is_the_sharded_sum(chunks):
    """oz_heff_apply_streamed on one GPU: the groups of the partition built, applied and released in
    turn give, bit for bit, the oracle's emulated product of every group summed in group order (for
    one chunk: the single handle's product)."""
    import paper_2510_04795_gb300 as oz
    ctx = oz.Context(0)
    st = synthetic.heff_structure(grid=(4, 4), dims=(8, 96), nterms=16, spread=True, seed=9)
    blocks = [tuple(b.cuda() for b in synthetic.gen_task_blocks(st, t)) for t in range(st.ntask)]
    psi = synthetic.gen_psi(st).cuda()
    tasks = [(int(s), int(d), float(st.term_coef[k]), L, R) for (k, s, d), (L, R) in zip(st.tasks, blocks)]
    Lb = [b[0].cpu().numpy() for b in blocks]
    Rb = [b[1].cpu().numpy() for b in blocks]
    psi_h = psi.cpu().numpy()
    y = oz.heff_apply_streamed(ctx, st.m, st.n, tasks, psi, chunks, slices=7)
    ctx.status()
    owner = oz.heff_partition(st.m, st.n, [t[0] for t in tasks], [t[1] for t in tasks], chunks)
    acc = None
    for r in range(chunks):
        ids = np.flatnonzero(owner == r)
        sub = synthetic.HeffStructure(st.labels, st.m, st.n, st.term_delta, st.term_coef, st.tasks[ids], st.spread,
                                      st.seed)
        ref = heff.heff_apply_emulated(sub, [Lb[i] for i in ids], [Rb[i] for i in ids], psi_h, 7)
        acc = ref if acc is None else acc + ref
    assert np.array_equal(y.cpu().numpy().view(np.int64), acc.view(np.int64))
    if chunks == 1:
        h = oz.Heff(ctx, st.m, st.n, tasks, slices=7)
        assert torch.equal(h.apply(psi), y)
        h.close()
    with pytest.raises(oz.OzError):
        oz.heff_apply_streamed(ctx, st.m, st.n, tasks, psi, 0)
    ctx.close()
