"""GPU parity of the audit quantities (probe information, reach, direct age
quantile, J_old) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=64, n_r=16, n_phi=32, n_frames=120, n_hats=32,
                     ss=2)
    tab = O.build_table(w, I.screen_samples(w))
    op = rtt.Operator(w, {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
                          "delay": tab.delay, "weight": tab.weight,
                          "throughput": tab.throughput})
    return w, tab, op


@pytest.mark.parametrize("mask", [1, 7])
def test_probe_info_matches_oracle(case, mask):
    w, tab, op = case
    sub = tab.select(tuple(n for n in range(3) if mask & (1 << n)))
    ref = O.probe_info(w, sub, O.scale(tab))
    got = rtt.probe_info(op, mask)
    big = ref > 1e-30 * ref.max()
    assert np.allclose(got[big], ref[big], rtol=2e-5)
    assert np.all(np.abs(got[~big]) <= 1e-6 * ref.max())
    # the pass/fail mask agrees wherever the oracle is not within 1e-9 of rho^2
    clear = np.abs(ref - 1.0) > 1e-9
    assert np.array_equal((got >= 1.0)[clear], (ref >= 1.0)[clear])


def test_reach_quantile_and_jold_match_oracle(case):
    w, tab, op = case
    scl = O.scale(tab)
    a0_ref = O.a0999(w, tab)
    a0 = rtt.direct_age_quantile(op, 0.999)
    assert a0 == pytest.approx(a0_ref, abs=1e-9)
    for mask, orders in ((1, (0,)), (7, (0, 1, 2))):
        info_ref = O.probe_info(w, tab.select(orders), scl)
        r_ref = O.reach(w, tab, info_ref, orders)
        info = rtt.probe_info(op, mask)
        res, passed = rtt.reach(op, info, mask, a0q=a0)
        assert np.array_equal(passed, r_ref.passing)
        assert (res.anchor_index >= 0) == (r_ref.anchor is not None)
        if r_ref.anchor is not None:
            assert res.anchor_age == r_ref.anchor
        assert res.L_anchor == r_ref.L_anchor
        assert res.J_old == pytest.approx(O.j_old(info_ref, a0_ref), rel=1e-5)


@pytest.mark.parametrize("kind", ["S224", "L224"])
def test_gram_eig_rank_match_oracle(kind):
    """Restricted Gram (FP64 path) and Jacobi spectrum vs the oracle on the
    Schwarzschild 32x32 workload, direct and resolved arms."""
    build.build()
    w = I.schw32()
    tab = O.build_table(w, I.screen_samples(w))
    op = rtt.Operator(w, {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
                          "delay": tab.delay, "weight": tab.weight,
                          "throughput": tab.throughput})
    scl = O.scale(tab)
    Q = O.synth_class(w, kind)
    Qd = torch.from_numpy(Q.reshape(w.grid.n_nodes, w.time.n_hats, -1).copy()).cuda()
    for mask, orders in ((1, (0,)), (7, (0, 1, 2))):
        P = O.restricted_response(w, tab.select(orders), Q, scl)
        G_ref = O.gram(P)
        G = rtt.gram(op, Qd, mask).cpu().numpy()
        Pg = op.apply_A(Qd, arm_mask=mask).reshape(-1, Q.shape[1])
        G_torch = (Pg.T @ Pg).cpu().numpy()
        err_p = np.max(np.abs(Pg.cpu().numpy() - P)) / np.max(np.abs(P))
        err_t = np.max(np.abs(G_torch - G_ref)) / np.max(np.abs(G_ref))
        loc = np.unravel_index(np.argmax(np.abs(G - G_ref)), G.shape)
        assert np.max(np.abs(G - G_ref)) <= 1e-12 * np.max(np.abs(G_ref)), (
            mask, err_p, err_t, loc, G[loc], G_ref[loc], G_torch[loc])
        ref = O.operational_rank(G_ref)
        sig, rank = rtt.operational_rank(op, Qd, mask)
        assert np.allclose(sig[:10], ref.sigma[:10], rtol=1e-10)
        lam_ref = ref.sigma ** 2
        lam = sig ** 2
        assert np.max(np.abs(lam - lam_ref)) <= 1e-11 * lam_ref[0]
        if ref.margin > 1e-6:
            assert rank == ref.rank


def test_ridge_cg_matches_oracle(case):
    """Batched ridge CG (FP32 with FP64 residual refresh) vs the oracle's FP64
    CG solution, for two histories x three regularisation values."""
    w, tab, op = case
    scl = O.scale(tab)
    xt = I.history_batch(w, [41, 42])
    data = O.apply_A(w, tab, xt, scl) + I.noise((tab.n_rows, w.time.n_frames, 2), 43)
    lams = [30.0, 300.0, 3000.0]
    x, iters, rel = rtt.solve_ridge(op, torch.from_numpy(data.astype(np.float32)).cuda(), lams,
                                    tol=1e-7, max_iter=4000, refresh_every=10)
    assert np.all(rel < 1e-6), rel
    xg = x.cpu().numpy()
    for j in range(2):
        for l, lam in enumerate(lams):
            ref, _ = O.ridge_cg(w, tab, scl, data[:, :, j:j + 1], lam, tol=1e-12)
            got = xg[:, :, j * len(lams) + l]
            err = np.linalg.norm(got - ref[:, :, 0]) / np.linalg.norm(ref)
            assert err < 1e-4, (j, lam, err)


def test_full_space_rank_32x32():
    """The 32x32 Schwarzschild workload audited on its full 1536-dimensional
    grid x hat space (Q = I): the restricted Gram through both FP64 routes,
    its eigenvalues (tridiagonal path) and the operational rank against the
    oracle's dense A, for the direct and resolved arms."""
    build.build()
    w = I.schw32()
    tab = O.build_table(w, I.screen_samples(w))
    op = rtt.Operator(w, {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
                          "delay": tab.delay, "weight": tab.weight,
                          "throughput": tab.throughput})
    scl = O.scale(tab)
    n = w.n_dof
    assert n == 1536
    Qd = torch.eye(n, dtype=torch.float64).reshape(w.grid.n_nodes, w.time.n_hats, n).cuda()
    for mask, orders in ((1, (0,)), (7, (0, 1, 2))):
        D = O.dense_A(w, tab.select(orders), scl)
        lam_ref = np.linalg.eigvalsh(D.T @ D)
        sig_ref = np.sqrt(np.maximum(lam_ref, 0.0))
        rank_ref = int(np.count_nonzero(sig_ref >= 1.0))
        margin = np.min(np.abs(sig_ref - 1.0))
        for mode in (rtt.GRAM_DATA, rtt.GRAM_NORMAL):
            G = rtt.gram(op, Qd, mask, mode=mode)
            ev = rtt.eigvals_sym_batched(G[None])[0]
            assert np.max(np.abs(ev - lam_ref)) <= 64 * n * 2.2e-16 * np.max(lam_ref) * 4
            sig = np.sqrt(np.maximum(ev, 0.0))
            if margin > 1e-6:
                assert int(np.count_nonzero(sig >= 1.0)) == rank_ref
        # blindness: the direct arm's rank is below the full dimension
        if mask == 1:
            assert rank_ref < n


def test_tsvd_matches_oracle():
    """TSVD in the S224 class truncated at the operational rank vs the oracle."""
    build.build()
    w = I.schw32()
    tab = O.build_table(w, I.screen_samples(w))
    op = rtt.Operator(w, {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
                          "delay": tab.delay, "weight": tab.weight,
                          "throughput": tab.throughput})
    scl = O.scale(tab)
    Q = O.synth_class(w, "S224")
    Qd = torch.from_numpy(Q.reshape(w.grid.n_nodes, w.time.n_hats, -1).copy()).cuda()
    xt = I.history_batch(w, [51, 52, 53])
    data = O.apply_A(w, tab, xt, scl) + I.noise((tab.n_rows, w.time.n_frames, 3), 54)
    ref, r_ref = O.tsvd_in_class(w, tab, scl, Q, data, None)
    G = rtt.gram(op, Qd, 7)
    ev, V, _ = rtt.eig_sym(G)
    rank = int(np.count_nonzero(np.sqrt(np.maximum(ev, 0)) >= 1.0))
    assert rank == r_ref
    xh = rtt.solve_tsvd(op, Qd, V, ev, rank, torch.from_numpy(data).cuda()).cpu().numpy()
    err = np.linalg.norm(xh - ref) / np.linalg.norm(ref)
    assert err < 1e-8, err


def test_gram_normal_operator_matches_oracle(case):
    """G = Q^T A^T A Q (normal-operator route, FP64) equals the oracle's P^T P."""
    w, tab, op = case
    scl = O.scale(tab)
    Q = O.synth_class(w, "S224")
    Qd = torch.from_numpy(Q.reshape(w.grid.n_nodes, w.time.n_hats, -1).copy()).cuda()
    for mask, orders in ((1, (0,)), (7, (0, 1, 2))):
        G_ref = O.gram(O.restricted_response(w, tab.select(orders), Q, scl))
        G = rtt.gram(op, Qd, mask, mode=rtt.GRAM_NORMAL).cpu().numpy()
        assert np.max(np.abs(G - G_ref)) <= 1e-11 * np.max(np.abs(G_ref))
        assert np.array_equal(G, G.T)


@pytest.mark.parametrize("kind", [0, 1])
def test_gram_class_matches_normal_and_oracle(case, kind):
    """rtt_gram_class (separable class, no P) equals the normal-operator Gram
    and the oracle's P^T P to FP64 rounding, for both arms."""
    w, tab, op = case
    scl = O.scale(tab)
    Q = O.synth_class(w, "S224" if kind == 0 else "L224")
    Qd = torch.from_numpy(Q.reshape(w.grid.n_nodes, w.time.n_hats, -1).copy()).cuda()
    for mask, orders in ((1, (0,)), (7, (0, 1, 2))):
        G_ref = O.gram(O.restricted_response(w, tab.select(orders), Q, scl))
        G = rtt.gram_class(op, kind, mask).cpu().numpy()
        Gn = rtt.gram(op, Qd, mask, mode=rtt.GRAM_NORMAL).cpu().numpy()
        assert np.array_equal(G, G.T)
        assert np.max(np.abs(G - G_ref)) <= 1e-11 * np.max(np.abs(G_ref))
        assert np.max(np.abs(G - Gn)) <= 1e-11 * np.max(np.abs(Gn))


def test_eigvals_tridiagonal_matches_numpy():
    """rtt_eigvals_sym_batched on graded symmetric matrices (eigenvalues from
    1e-2 to 1e11, as the restricted Grams): every eigenvalue within
    64 n eps max|lambda| of numpy's, the largest ones to 1e-11 relative."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    rng = np.random.default_rng(8)
    n, b = 96, 5
    mats = []
    for _ in range(b):
        Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = 10.0 ** rng.uniform(-2, 11, n)
        A = (Qm * lam) @ Qm.T
        mats.append(0.5 * (A + A.T))
    G = torch.from_numpy(np.stack(mats)).cuda()
    ev = rtt.eigvals_sym_batched(G)
    for i in range(b):
        ref = np.linalg.eigvalsh(mats[i])
        bound = 64 * n * 2.2e-16 * np.max(np.abs(ref))
        assert np.max(np.abs(ev[i] - ref)) <= bound
        big = ref > 1e-2 * ref.max()
        assert np.max(np.abs(ev[i][big] / ref[big] - 1.0)) <= 1e-11


def test_rank_audit_matches_oracle():
    """rtt_rank_audit over two geometries and two arms: rank, reach, J_old and
    A_0.999 against the oracle's audit of the same tables."""
    build.build()
    ws = [I.small_kerr(spin=0.0, incl_deg=20.0, nx=40, n_r=10, n_phi=20, n_frames=80, n_hats=20),
          I.small_kerr(spin=0.5, incl_deg=50.0, nx=40, n_r=10, n_phi=20, n_frames=80, n_hats=20)]
    ops, Qs, refs = [], [], []
    for w in ws:
        tab = O.build_table(w, I.screen_samples(w))
        ops.append(rtt.Operator(w, {"order": tab.order, "pixel": tab.pixel, "r": tab.r,
                                    "phi": tab.phi, "delay": tab.delay, "weight": tab.weight,
                                    "throughput": tab.throughput}))
        Q = O.synth_class(w, "S224")
        Qs.append(torch.from_numpy(Q.reshape(w.grid.n_nodes, w.time.n_hats, -1).copy()).cuda())
        scl = O.scale(tab)
        a0 = O.a0999(w, tab)
        per_arm = []
        for orders in ((0,), (0, 1, 2)):
            info = O.probe_info(w, tab.select(orders), scl)
            rr = O.reach(w, tab, info, orders)
            spec = O.operational_rank(O.gram(O.restricted_response(w, tab.select(orders), Q, scl)))
            per_arm.append((rr, O.j_old(info, a0), spec, a0))
        refs.append(per_arm)
    for mode in (rtt.GRAM_DATA, rtt.GRAM_NORMAL, rtt.GRAM_CLASS_S224):
        recs, sig = rtt.rank_audit(ops, None if mode == rtt.GRAM_CLASS_S224 else Qs, (1, 7),
                                   mode=mode)
        for g in range(2):
            for a in range(2):
                rr, jo, spec, a0 = refs[g][a]
                r = recs[g][a]
                if spec.margin > 1e-6:
                    assert r.rank == spec.rank
                assert np.allclose(sig[g, a, :10], spec.sigma[:10], rtol=1e-9)
                assert r.reach.L_anchor == rr.L_anchor
                assert r.reach.A0q == pytest.approx(a0, abs=1e-9)
                assert r.reach.J_old == pytest.approx(jo, rel=1e-5)


@pytest.mark.parametrize("kind", [0, 1])
def test_class_synthesis_matches_oracle(case, kind):
    w, tab, op = case
    Q_ref = O.synth_class(w, "S224" if kind == 0 else "L224")
    Q = rtt.synth_class(op, kind).cpu().numpy().reshape(Q_ref.shape)
    assert np.max(np.abs(Q - Q_ref)) <= 1e-13
