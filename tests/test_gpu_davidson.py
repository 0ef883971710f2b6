"""GPU Davidson (davidson_start/step/ritz/solve, oz_heff_diag, oz_symeig_small) against the oracle
Davidson and dense numpy eigensolutions of the same H_eff."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import davidson as odav
from oracle import heff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2510_04795_gb300 as oz
    c = oz.Context(0)
    yield c
    c.close()


def _problem(grid, dims, nterms, spread, seed):
    st = synthetic.heff_structure(grid=grid, dims=dims, nterms=nterms, spread=spread, seed=seed)
    blocks = [synthetic.gen_task_blocks(st, t, device="cuda") for t in range(st.ntask)]
    psi = synthetic.gen_psi(st, device="cuda")
    tasks = [(int(s), int(d), float(st.term_coef[k]), L, R) for (k, s, d), (L, R) in zip(st.tasks, blocks)]
    Lb = [b[0].cpu().numpy() for b in blocks]
    Rb = [b[1].cpu().numpy() for b in blocks]
    return st, tasks, Lb, Rb, psi


@pytest.mark.parametrize("m", [1, 2, 3, 7, 16, 24, 31, 32])
def test_symeig_small_random(m):
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(m)
    A = rng.normal(size=(m, m))
    A = A + A.T
    w, V = oz.symeig_small(torch.from_numpy(A).cuda())
    w, V = w.cpu().numpy(), V.cpu().numpy()
    nrm = np.linalg.norm(A)
    assert np.allclose(w, np.linalg.eigvalsh(A), rtol=0, atol=1e-13 * nrm)
    assert np.all(np.diff(w) >= 0)
    assert np.linalg.norm(A @ V - V * w) <= 1e-13 * nrm
    assert np.linalg.norm(V.T @ V - np.eye(m)) <= 1e-13 * m


def test_symeig_small_degenerate_and_special():
    import paper_2510_04795_gb300 as oz
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.normal(size=(12, 12)))
    lam = np.array([-3.0, -3.0, -3.0, 0.0, 0.0, 1.0, 2.0, 2.0, 5.0, 7.0, 7.0, 9.0])
    cases = [Q @ np.diag(lam) @ Q.T, np.diag(rng.normal(size=9)), np.zeros((5, 5)),
             np.array([[1e-300, 0.0], [0.0, -1e-300]]), np.array([[2.0, 1e-20], [1e-20, 2.0]])]
    for A in cases:
        A = 0.5 * (A + A.T)
        w, V = oz.symeig_small(torch.from_numpy(A.copy()).cuda())
        w, V = w.cpu().numpy(), V.cpu().numpy()
        nrm = max(np.linalg.norm(A), 1e-300)
        assert np.allclose(w, np.linalg.eigvalsh(A), rtol=0, atol=1e-13 * nrm)
        assert np.linalg.norm(A @ V - V * w) <= 1e-13 * nrm
        assert np.linalg.norm(V.T @ V - np.eye(len(A))) <= 1e-12


def test_heff_diag_matches_oracle(ctx):
    import paper_2510_04795_gb300 as oz
    st, tasks, Lb, Rb, psi = _problem((4, 3), (5, 40), 12, True, 21)
    for mode in ("eager", "native"):
        h = oz.Heff(ctx, st.m, st.n, tasks, slices=7, mode=mode)
        got = h.diag().cpu().numpy()
        ref = heff.heff_diag(st, Lb, Rb)
        # rounding bound of a sum of products: a few ulps of the sum of their magnitudes
        off = st.psi_offsets()
        mag = np.zeros_like(ref)
        for t, (k, s, d) in enumerate(st.tasks):
            if s == d:
                blk = abs(st.term_coef[k]) * np.outer(np.abs(np.diag(Lb[t])), np.abs(np.diag(Rb[t])))
                mag[off[s]:off[s + 1]] += blk.reshape(-1)
        assert np.all(np.abs(got - ref) <= 8 * np.finfo(float).eps * mag)
        assert np.count_nonzero(ref) > 0
        h.close()


@pytest.mark.parametrize("mode", ["eager", "native"])
def test_davidson_solve_vs_dense_eigh(ctx, mode):
    import paper_2510_04795_gb300 as oz
    st, tasks, Lb, Rb, psi = _problem((3, 3), (3, 14), 10, False, 22)
    H = heff.heff_dense(st, Lb, Rb)
    assert H.shape[0] <= 3000
    lam, U = np.linalg.eigh(H)
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=7, mode=mode)
    x = psi.clone()
    e, it, rc = oz.davidson_solve(h, x, tol=1e-10, max_iter=400)
    ctx.status()
    assert rc == 0 and it > 1
    assert abs(e - lam[0]) <= 1e-9 * max(1.0, abs(lam[0]))
    xv = x.cpu().numpy()
    assert abs(np.linalg.norm(xv) - 1.0) < 1e-12
    gap = lam[1] - lam[0]
    assert abs(abs(xv @ U[:, 0]) - 1.0) <= max(1e-12, 4 * (1e-10 / gap) ** 2)
    # the returned vector is an eigenvector of the FP64 operator to the residual tolerance
    assert np.linalg.norm(H @ xv - e * xv) <= 1e-9 * max(1.0, abs(e))
    h.close()


@pytest.mark.parametrize("mode", ["eager", "native"])
def test_davidson_steps_follow_oracle(ctx, mode):
    """Same start vector, same algorithm: the Ritz values of every iteration agree with the oracle
    Davidson (FP64 numpy products) far below the residual tolerance, and both stop together."""
    import paper_2510_04795_gb300 as oz
    st, tasks, Lb, Rb, psi = _problem((4, 4), (6, 48), 16, False, 23)
    hist = []
    diag = heff.heff_diag(st, Lb, Rb)
    th_o, x_o, it_o, ok = odav.davidson(lambda v: heff.heff_apply_fp64(st, Lb, Rb, v), diag, psi.cpu().numpy(),
                                        tol=1e-10, max_iter=300, max_sub=24, history=hist)
    assert ok
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=7, mode=mode)
    dv = oz.Davidson(h, max_sub=24, tol=1e-10)
    dv.start(psi)
    got = []
    while True:
        th, rs, cv = dv.step()
        got.append((th, rs))
        if cv or len(got) >= 300:
            break
    ctx.status()
    assert cv
    assert abs(len(got) - it_o) <= max(3, it_o // 10)
    n = min(len(got), len(hist))
    hn = abs(th_o)   # the spectral radius scale: product errors are relative to |H|, not to theta
    for i, ((a, ra), (b, rb)) in enumerate(zip(got[:n], hist[:n])):
        # two Ritz values whose residuals are ra and rb lie within (ra^2 + rb^2)/gap of the same
        # eigenvalue; the gap of this spectrum is O(1)
        assert abs(a - b) <= 1e-10 * hn + 2.0 * (ra * ra + rb * rb)
        if i < 2:   # the first subspaces are the same up to rounding; later the preconditioner
            #          1/(theta - diag) amplifies rounding differences between the two products
            assert abs(a - b) <= 1e-13 * hn
            assert abs(ra - rb) <= 1e-10 * hn
    x = dv.ritz().cpu().numpy()
    assert abs(abs(x @ x_o) - 1.0) < 1e-12
    dv.close()
    h.close()


def test_davidson_restart_small_subspace(ctx):
    import paper_2510_04795_gb300 as oz
    st, tasks, Lb, Rb, psi = _problem((3, 3), (3, 14), 10, False, 22)
    H = heff.heff_dense(st, Lb, Rb)
    lam = np.linalg.eigvalsh(H)
    hist = []
    th_o, _, it_o, ok = odav.davidson(lambda v: H @ v, np.diag(H), psi.cpu().numpy(), tol=1e-9, max_iter=600,
                                      max_sub=6, history=hist)
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=7)
    dv = oz.Davidson(h, max_sub=6, tol=1e-9)
    dv.start(psi)
    seq = []
    for _ in range(600):
        th, rs, cv = dv.step()
        seq.append(th)
        if cv:
            break
    assert cv and len(seq) > 6               # restarts happened
    assert abs(seq[-1] - lam[0]) <= 1e-8 * abs(lam[0])
    assert all(b <= a + 1e-10 * abs(a) for a, b in zip(seq, seq[1:]))  # Ritz values never rise
    if ok:
        assert abs(len(seq) - it_o) <= max(3, it_o // 10)
    dv.close()
    h.close()


def test_davidson_status_codes(ctx):
    import paper_2510_04795_gb300 as oz
    from paper_2510_04795_gb300 import OzError
    st, tasks, Lb, Rb, psi = _problem((3, 2), (3, 10), 6, False, 24)
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=7)
    x = psi.clone()
    e, it, rc = oz.davidson_solve(h, x, tol=1e-14, max_iter=2)
    assert rc == 3 and it == 2 and np.isfinite(e)           # OZ_ENOCONV, last iterate returned
    assert abs(torch.linalg.norm(x).item() - 1.0) < 1e-12
    dv = oz.Davidson(h, max_sub=8, tol=1e-10)
    with pytest.raises(OzError):
        dv.start(torch.zeros_like(psi))                     # zero start vector: OZ_EINVAL
    with pytest.raises(OzError):
        oz.Davidson(h, max_sub=2)                           # subspace too small
    dv.close()
    h.close()


@pytest.mark.parametrize("krylov", [30, 8])
def test_lanczos_vs_oracle_and_eigh(ctx, krylov):
    """Device Lanczos (full reorthogonalisation, explicit restarts every `krylov` vectors) against
    dense eigh and against the oracle Lanczos on the same operator."""
    import paper_2510_04795_gb300 as oz
    from oracle import lanczos as olz
    st, tasks, Lb, Rb, psi = _problem((3, 3), (3, 14), 10, False, 22)
    H = heff.heff_dense(st, Lb, Rb)
    lam, U = np.linalg.eigh(H)
    h = oz.Heff(ctx, st.m, st.n, tasks, slices=7)
    x = psi.clone()
    e, it, rc = oz.lanczos_solve(h, x, eps=1e-10, max_iter=2000, krylov=krylov)
    assert rc == 0
    assert abs(e - lam[0]) <= 1e-9 * abs(lam[0])
    xv = x.cpu().numpy()
    assert abs(abs(xv @ U[:, 0]) - 1.0) <= 1e-9
    th, xo, it_o, ok = olz.lanczos(lambda v: H @ v, psi.cpu().numpy(), eps=1e-10, max_iter=2000, krylov=krylov)
    assert ok and abs(th - e) <= 1e-9 * abs(lam[0])
    assert abs(it - it_o) <= max(3, it_o // 10)
    h.close()
