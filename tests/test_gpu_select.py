"""The per-block precision dial and its learned selector: the network's gradients against the
oracle, the harvested errors against the oracle's emulated products, and what the trained
network gains over a fixed slice count at the same error budget."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import heff as oheff
from oracle import mlp as omlp
from oracle import ozaki

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_04795_gb300 as oz
    c = oz.Context(0)
    yield c
    c.close()


def _structure(seed, grid=(5, 4), dims=(8, 96), nterms=24, decades=6.0):
    st = synthetic.heff_structure(grid=grid, dims=dims, nterms=nterms, spread=True, seed=seed, widths=True)
    blocks = [synthetic.gen_task_blocks(st, t, device="cuda") for t in range(st.ntask)]
    tasks = [(int(s), int(d), float(st.term_coef[k]), L, R) for (k, s, d), (L, R) in zip(st.tasks, blocks)]
    psi = synthetic.gen_psi(st, seed=seed + 1000, device="cuda", decades=decades)
    return st, blocks, tasks, psi


def test_mlp_gradient_matches_oracle():
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(0)
    net = oz.MLP(nin=20, nhidden=64, nout=6, seed=7)
    flat = net.params().astype(np.float64)
    X = rng.normal(size=(57, 20)).astype(np.float32)
    T = rng.normal(size=(57, 6)).astype(np.float32)
    M = (rng.uniform(size=(57, 6)) < 0.7).astype(np.float32)
    loss, g = net.gradient(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(M).cuda())
    ref_loss, ref_g = omlp.loss_and_grads(omlp.unflatten(flat, 20, 64, 6), X.astype(np.float64),
                                          T.astype(np.float64), M.astype(np.float64))
    ref_g = omlp.flatten(ref_g)
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss)
    assert np.max(np.abs(g - ref_g)) <= 1e-4 * np.max(np.abs(ref_g))
    Y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    Yref, _ = omlp.forward(omlp.unflatten(flat, 20, 64, 6), X.astype(np.float64))
    assert np.max(np.abs(Y - Yref)) <= 1e-5 * max(1.0, np.max(np.abs(Yref)))
    net.close()


def test_mlp_training_reproducible_and_converging():
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(1)
    X = rng.normal(size=(512, 20)).astype(np.float32)
    W = rng.normal(size=(20, 6)).astype(np.float32)
    T = np.tanh(X @ W) * 3.0 - 8.0
    M = np.ones_like(T)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    params = []
    for _ in range(2):
        net = oz.MLP(seed=11)
        l0 = net.gradient(d(X), d(T), d(M))[0]
        loss = net.train(d(X), d(T), d(M), epochs=60, batch=64, lr=2e-3, seed=3)
        params.append(net.params())
        net.close()
    assert np.array_equal(params[0], params[1])
    assert loss < 0.05 * l0


def test_problem_errors_match_oracle(ctx):
    """The harvested per-product errors are the errors of the oracle's emulated products."""
    import paper_2510_04795_gb300 as oz
    st, blocks, tasks, psi = _structure(41, grid=(3, 3), dims=(4, 24), nterms=6, decades=3.0)
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=9, level=8)
    e1, e2 = h.problem_errors(psi, 4)
    Lb = [b[0].cpu().numpy() for b in blocks]
    Rb = [b[1].cpu().numpy() for b in blocks]
    P = psi.cpu().numpy()
    off = st.psi_offsets()
    by_src, by_dst = oheff.emulated_groups(st)
    Tfull = {}
    for q in range(st.nsec):
        if not by_src[q]:
            assert e1[q] == -1.0
            continue
        A1 = np.vstack([Lb[t] for t in by_src[q]])
        Bq = P[off[q]:off[q + 1]].reshape(st.m[q], st.n[q])
        ref = ozaki.ozaki_gemm(A1, Bq, 9, 8)
        got = ozaki.ozaki_gemm(A1, Bq, 9, 4)
        want = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert abs(e1[q] - want) <= 1e-9 * want
        r = 0
        for t in by_src[q]:
            Tfull[t] = ref[r:r + Lb[t].shape[0]]
            r += Lb[t].shape[0]
    for q in range(st.nsec):
        if not by_dst[q]:
            continue
        A2 = np.hstack([Tfull[t] for t in by_dst[q]])
        B2 = np.vstack([(st.term_coef[st.tasks[t][0]] * Rb[t]).T for t in by_dst[q]])
        ref = ozaki.ozaki_gemm(A2, B2, 9, 8)
        got = ozaki.ozaki_gemm(A2, B2, 9, 4)
        want = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert abs(e2[q] - want) <= 1e-9 * want
    h.close()


def test_learned_selector_meets_budget_with_fewer_flops(ctx):
    """Trained on (features, measured error) pairs harvested from 40 structures, the network picks
    per-product levels for 6 unseen structures that keep H_eff psi within the 1e-12 budget with
    fewer carrier flops than the fixed slice count 7, than the analytic selector and than the best
    uniform level chosen in hindsight."""
    import paper_2510_04795_gb300 as oz
    from paper_2510_04795_gb300 import selector
    rows = []
    for sd in range(100, 140):
        st, blocks, tasks, psi = _structure(sd)
        h = oz.Heff(ctx, st.m, st.n, tasks, slices=9, level=8)
        rows.append(selector.harvest(h, psi))
        h.close()
    X, T, M = (np.concatenate([r[i] for r in rows]) for i in range(3))
    net = selector.train(X, T, M, epochs=400, batch=64, lr=2e-3, seed=4)
    budget = 1e-12
    tot = {"fixed7": 0, "analytic": 0, "learned": 0, "uniform": 0}
    for sd in range(300, 306):
        st, blocks, tasks, psi = _structure(sd)
        h = oz.Heff(ctx, st.m, st.n, tasks, slices=9, level=8)
        yref = h.apply(psi).clone()
        err = lambda: (torch.linalg.norm(h.apply(psi) - yref) / torch.linalg.norm(yref)).item()
        for lev in range(3, 9):                      # best uniform level, in hindsight
            h.set_levels([lev] * st.nsec, [lev] * st.nsec)
            if err() <= budget:
                break
        tot["uniform"] += h.info()["carrier_flops"]
        h.set_levels([7] * st.nsec, [7] * st.nsec)
        assert err() <= budget
        tot["fixed7"] += h.info()["carrier_flops"]
        for name in ("analytic", "learned"):
            h.select_levels(psi, selector=name, budget=budget, net=net, margin=0.3)
            e = err()
            assert e <= budget, (sd, name, e)
            tot[name] += h.info()["carrier_flops"]
        h.close()
    assert tot["learned"] <= 0.8 * tot["fixed7"]
    assert tot["learned"] < tot["analytic"]
    assert tot["learned"] < tot["uniform"]
    net.close()
