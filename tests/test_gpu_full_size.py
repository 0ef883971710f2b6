"""H_eff psi at the full size of the timed workload, in the launch configuration the bench times.

300 sector blocks of 16-1024, 200 terms, S = 7 (54,688 tasks, 136 GB of operator digit planes):
the whole product runs on the GPU with the autotuned tile schedules and the captured graph, and
sampled entries are compared bit for bit with the oracle's emulated definition, computed entry by
entry (``oracle.heff.heff_entries_emulated``) from the operand rows the device used.  The samples
cover eight cheap target sectors (both stage-2 orientations), the target sector with the longest
stage-2 reduction (the most accumulator groups and drains per diagonal) and a target sector fed by
the largest stage-1 source block, each at a random and the last row and column.
"""
import numpy as np
import pytest

import synthetic
from oracle import heff

pytestmark = pytest.mark.gpu


def _cheap_targets(st, count):
    # target sectors whose source blocks the CPU oracle slices in about a second
    m, n, T = st.m.astype(np.int64), st.n.astype(np.int64), st.tasks
    cost = []
    for q in range(st.nsec):
        srcs = np.unique(T[T[:, 2] == q][:, 1])
        if srcs.size:
            cost.append((int((m[srcs] * n[srcs]).sum()), q))
    cost.sort()
    return [q for _, q in cost[:count]]


def _stage2_k(st, q):
    # length of the stage-2 reduction of target q: the concatenated columns of its T blocks
    T = st.tasks
    return int(st.n[T[T[:, 2] == q][:, 1]].sum())


def test_full_workload_sampled_entries_bitexact():
    import torch
    import paper_2510_04795_gb300 as oz
    st = synthetic.heff_structure(**synthetic.CONFIGS["heff300_16-1024"])
    torch.cuda.empty_cache()
    ctx = oz.Context(0)
    Lbuf, Rbuf, Lo, Ro = synthetic.gen_all_task_blocks(st, device="cuda")
    psi = synthetic.gen_psi(st, device="cuda")
    tasks = []
    for t, (k, s, d) in enumerate(st.tasks):
        L = Lbuf[Lo[t]:Lo[t + 1]].view(int(st.m[d]), int(st.m[s]))
        R = Rbuf[Ro[t]:Ro[t + 1]].view(int(st.n[d]), int(st.n[s]))
        tasks.append((int(s), int(d), float(st.term_coef[k]), L, R))
    # sampled entries: a random row and the last row, a random column and the last column
    rng = np.random.default_rng(11)
    picks = []
    cheap = _cheap_targets(st, 8)
    k2 = [_stage2_k(st, q) for q in range(st.nsec)]
    longest = int(np.argmax(k2))
    big_src = int(np.argmax(st.m.astype(np.int64) * st.n.astype(np.int64)))
    fed = sorted({int(d) for (_, s_, d) in st.tasks if int(s_) == big_src} - {longest} - set(cheap))
    assert k2[longest] >= 20000 and fed
    targets = cheap + [longest, fed[0]]
    for q in targets:
        mq, nq = int(st.m[q]), int(st.n[q])
        js = sorted({int(rng.integers(nq)), nq - 1})
        for i in sorted({int(rng.integers(mq)), mq - 1}):
            picks.append((q, i, js))
    # host copies of the operand rows those entries depend on
    off = st.psi_offsets()
    psi_h = psi.cpu().numpy()
    need = {}
    for q, i, js in picks:
        into = [t for t in range(st.ntask) if int(st.tasks[t][2]) == q]
        L_rows = {t: tasks[t][3][i].cpu().numpy() for t in into}
        R_rows = {t: tasks[t][4][js].cpu().numpy() for t in into}
        P = {}
        for t in into:
            s = int(st.tasks[t][1])
            P[s] = psi_h[off[s]:off[s + 1]].reshape(int(st.m[s]), int(st.n[s]))
        need[(q, i)] = (L_rows, R_rows, P)
    swapped = sum(1 for q in set(cheap)
                  if -(-int(st.n[q]) // 128) * 128 * -(-int(st.m[q]) // 64) * 64
                  < -(-int(st.m[q]) // 128) * 128 * -(-int(st.n[q]) // 64) * 64)
    assert 0 < swapped < len(cheap)  # both stage-2 orientations are sampled

    h = oz.Heff(ctx, st.m, st.n, tasks, slices=7)
    del tasks, Lbuf, Rbuf
    torch.cuda.empty_cache()
    h.autotune(psi, reps=1)
    y = h.apply(psi)
    ctx.status()
    y_h = y.cpu().numpy()
    h.close()
    ctx.close()
    for q, i, js in picks:
        L_rows, R_rows, P = need[(q, i)]
        ref = heff.heff_entries_emulated(st, q, i, js, L_rows, R_rows, P, 7)
        got = y_h[off[q] + i * int(st.n[q]) + np.array(js)]
        assert np.array_equal(got, ref), (q, i, js, got, ref)
