"""Term-sharded H_eff psi on CPU ranks: the host partition of the library (oz_heff_partition) and
the gather + rank-ordered sum of the partial products over torch.distributed with gloo, world
size 2.  The partial products come from the oracle (no GPU here); the GPU side of the same split
is tests/test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synthetic


def _struct():
    return synthetic.heff_structure(grid=(3, 3), dims=(4, 40), nterms=12, spread=True, seed=5)


def _sub(st, ids):
    return synthetic.HeffStructure(st.labels, st.m, st.n, st.term_delta, st.term_coef, st.tasks[ids], st.spread,
                                   st.seed)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_partition_owns_every_task_once_and_balances(world):
    import paper_2510_04795_gb300 as oz
    st = synthetic.heff_structure(**synthetic.CONFIGS["heff300_16-1024"])
    src, dst = st.tasks[:, 1], st.tasks[:, 2]
    own = oz.heff_partition(st.m, st.n, src, dst, world)
    assert own.shape == (st.ntask,) and own.min() >= 0 and own.max() < world
    assert np.array_equal(own, oz.heff_partition(st.m, st.n, src, dst, world))    # deterministic
    m, n = st.m.astype(np.int64), st.n.astype(np.int64)
    cost = 2 * m[dst] * m[src] * n[src] + 2 * m[dst] * n[src] * n[dst]
    load = np.bincount(own, weights=cost, minlength=world)
    assert load.sum() == cost.sum()
    # longest-first greedy: no rank exceeds the lightest by more than one task's cost
    assert load.max() - load.min() <= cost.max()


def test_partition_rejects_bad_arguments():
    import paper_2510_04795_gb300 as oz
    from paper_2510_04795_gb300 import OzError
    with pytest.raises(OzError):
        oz.heff_partition([2, 3], [2, 3], [0], [1], 0)
    with pytest.raises(OzError):
        oz.heff_partition([2, 3], [2, 3], [0], [2], 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2510_04795_gb300 as oz
    from oracle import heff
    st = _struct()
    Lb, Rb = [], []
    for t in range(st.ntask):
        L, R = synthetic.gen_task_blocks(st, t)
        Lb.append(L.numpy())
        Rb.append(R.numpy())
    psi = synthetic.gen_psi(st).numpy()
    own = oz.heff_partition(st.m, st.n, st.tasks[:, 1], st.tasks[:, 2], world)
    ids = np.nonzero(own == rank)[0]
    sub = _sub(st, ids)
    parts = {}
    for name, fn in (("fp64", lambda: heff.heff_apply_fp64(sub, [Lb[i] for i in ids], [Rb[i] for i in ids], psi)),
                     ("emul", lambda: heff.heff_apply_emulated(sub, [Lb[i] for i in ids], [Rb[i] for i in ids], psi,
                                                               7))):
        mine = torch.from_numpy(np.ascontiguousarray(fn()))
        gathered = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(gathered, mine)
        y = gathered[0].clone()
        for r in range(1, world):
            y = y + gathered[r]                     # rank order, one rounding per addition
        parts[name] = y.numpy()
    if rank == 0:
        out["fp64"] = parts["fp64"]
        out["emul"] = parts["emul"]
        out["ref64"] = heff.heff_apply_fp64(st, Lb, Rb, psi)
        out["refemul"] = heff.heff_apply_emulated(st, Lb, Rb, psi, 7)
        out["owned"] = int(len(ids))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_sum_over_gloo_ranks():
    """World size 2: each rank computes the partial product of its own tasks, the partial vectors
    are gathered and summed in rank order.  FP64 partials reproduce the unsharded FP64 product to
    rounding (1e-14 relative); emulated partials at S = 7 reproduce the unsharded emulated product
    within 1e-13 relative -- the stage-2 exponents of a target sector are shared only by the
    tasks on the same rank, so the two differ in the last bits, not bit for bit."""
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert 0 < out["owned"] < _struct().ntask
    assert rel(out["fp64"], out["ref64"]) <= 1e-14
    assert rel(out["emul"], out["refemul"]) <= 1e-13
    assert rel(out["emul"], out["ref64"]) <= 1e-12
