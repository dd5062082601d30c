"""Pins of the oracle's operator, whitening, probes, reach, classes, rank and
estimators against brute force, invariants and the paper's exact results."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O
from paper_2609_05528_b300 import inputs as I


@pytest.fixture(scope="module")
def schw():
    w = I.schw32()
    tab = O.build_table(w, I.screen_samples(w))
    return w, tab


@pytest.fixture(scope="module")
def tiny_kerr():
    w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=20, n_r=5, n_phi=8, n_frames=14, n_hats=6, ss=2)
    tab = O.build_table(w, I.screen_samples(w))
    return w, tab


def test_dense_assembly_matches_matrix_free(tiny_kerr):
    """Explicit per-ray assembly (numpy) == matrix-free C apply on unit vectors."""
    w, tab = tiny_kerr
    assert tab.rows_of_order(1) > 0
    D = O.dense_A(w, tab, 2.5)
    n = w.n_dof
    E = np.eye(n).reshape(w.grid.n_nodes, w.time.n_hats, n)
    M = O.apply_A(w, tab, E, 2.5).reshape(-1, n)
    assert np.max(np.abs(D - M)) <= 1e-15 * np.max(np.abs(D))
    # the adjoint applied to unit data vectors gives the transposed matrix
    m = tab.n_rows * w.time.n_frames
    Y = np.eye(m).reshape(tab.n_rows, w.time.n_frames, m)
    MT = O.apply_AT(w, tab, Y, 2.5).reshape(n, m)
    assert np.max(np.abs(MT - D.T)) <= 1e-15 * np.max(np.abs(D))


@pytest.mark.parametrize("which", ["schw", "tiny_kerr"])
def test_dot_product(which, request):
    """<A x, y> = <x, A^T y> to 1e-12."""
    w, tab = request.getfixturevalue(which)
    x = I.uniform_batch(w, [11, 12])
    y = I.noise((tab.n_rows, w.time.n_frames, 2), 13)
    Ax = O.apply_A(w, tab, x, 3.0)
    Aty = O.apply_AT(w, tab, y, 3.0)
    lhs = np.sum(Ax * y)
    rhs = np.sum(x * Aty)
    assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(Ax * Ax) * np.sum(y * y))


def test_single_ray_hand_computed():
    """One ray on a node, at a hat centre: y = w x[node][k] exactly; half way
    between two hats: the average of the two."""
    w = I.Workload("hand", I.Geometry(0.0, 20.0, 4), I.SourceGrid(3, 4, 3.0, 12.0),
                   I.TimeGrid(3, 2.0, 4, t_end=4.0))
    r_mid = 6.0  # log-spaced nodes 3, 6, 12
    tab = O.Table(np.array([0], np.int8), np.array([0], np.int32), np.array([r_mid]),
                  np.array([math.pi / 2]), np.array([0.0]), np.array([0.7]), np.array([1.0]),
                  np.array([0, 1], np.int64), np.array([0], np.int8), np.array([0], np.int32),
                  np.array([0], np.int64))
    x = np.zeros((w.grid.n_nodes, w.time.n_hats))
    node = 1 * 4 + 1  # r index 1, phi index 1 (= pi/2)
    x[node, :] = [10.0, 20.0, 30.0, 40.0]  # t_k = 4, 0, -4, -8
    y = O.apply_A(w, tab, x, 1.0)
    # frames t = 0, 2, 4 -> source times 0, 2, 4 -> hats k=1 (t=0), mid(0,1), k=0
    assert y[0, 0] == pytest.approx(0.7 * 20.0, rel=1e-15)
    assert y[0, 1] == pytest.approx(0.7 * 15.0, rel=1e-15)
    assert y[0, 2] == pytest.approx(0.7 * 10.0, rel=1e-15)


def _split_samples(s: I.ScreenSamples) -> I.ScreenSamples:
    """Every pixel split into 4 equal-area children with identical transfer
    values (the same screen point), each a pixel of its own."""
    idx = np.repeat(np.arange(len(s)), 4)
    child = np.tile(np.arange(4), len(s))
    return I.ScreenSamples(s.alpha[idx], s.beta[idx], (s.pixel[idx] * 4 + child).astype(np.int32),
                           s.n_sub[idx], s.d_omega_pixel / 4.0)


def test_split_merge_gram_invariance(paper):
    """Sec. 3.4: splitting pixels into equal-area children with identical
    transfer values leaves the Gram matrix unchanged (< 1e-10 relative)."""
    w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=16, n_r=4, n_phi=8, n_frames=10, n_hats=5, ss=2)
    s = I.screen_samples(w)
    t1 = O.build_table(w, s)
    t2 = O.build_table(w, _split_samples(s))
    G1 = O.dense_A(w, t1).T @ O.dense_A(w, t1)
    G2 = O.dense_A(w, t2).T @ O.dense_A(w, t2)
    rel = np.linalg.norm(G1 - G2) / np.linalg.norm(G1)
    assert rel < paper["split_merge_criterion"]
    # the SNR normalisation is split-invariant too (Eq. 17)
    assert O.s_ref(t2) == pytest.approx(O.s_ref(t1) / 2.0, rel=1e-12)


def test_gram_monotone_in_orders(tiny_kerr):
    """Eq. 21 / Eq. 46: G_{0:2} - G_0 is positive semidefinite."""
    w, tab = tiny_kerr
    G0 = O.dense_A(w, tab.select((0,))).T @ O.dense_A(w, tab.select((0,)))
    G = O.dense_A(w, tab).T @ O.dense_A(w, tab)
    ev = np.linalg.eigvalsh(G - G0)
    assert ev.min() >= -1e-12 * np.linalg.norm(G, 2)
    assert ev.max() > 0


def test_direct_old_epoch_blindness(schw, paper):
    """Theorem 4.1 / Cor. 4.2: hats whose support misses the discrete direct
    footprint W_0 (Eq. 23) give bit-identically zero direct columns for every
    node; the resolved stack lifts some of them; each hat that meets W_0 has
    a nonzero direct column."""
    w, tab = schw
    t = w.time
    K, S = t.n_hats, w.grid.n_nodes
    D0 = O.dense_A(w, tab.select((0,)))
    D = O.dense_A(w, tab)
    to = t.frame_times()
    W0 = (to[None, :] - tab.delay[tab.order == 0][:, None]).ravel()
    Wall = (to[None, :] - tab.delay[:, None]).ravel()
    tk = t.hat_times()
    missing = [k for k in range(K) if not np.any(np.abs(W0 - tk[k]) < t.hat_step)]
    assert len(missing) >= 2
    for k in range(K):
        cols = D0[:, [s * K + k for s in range(S)]]
        if k in missing:
            assert np.all(cols == 0.0)
        else:
            assert np.any(cols != 0.0)
    zero0 = np.all(D0 == 0.0, axis=0).reshape(S, K)
    assert zero0[:, missing].all()
    assert int(zero0.sum()) >= len(missing) * S
    # resolved stack: a missing direct hat whose support meets W_1 is lifted
    lifted = [k for k in missing if np.any(np.abs(Wall - tk[k]) < t.hat_step)]
    assert lifted
    for k in lifted:
        assert np.any(D[:, [s * K + k for s in range(S)]] != 0.0)
    # compact class L224: zero direct columns = (missing temporal factors) x 28
    Q = O.synth_class(w, "L224")
    P0 = D0 @ Q
    zc = np.all(P0 == 0.0, axis=0)
    tau = Q.reshape(S, K, 4, 7, 8)[0, :, 0, 0, :] / Q.reshape(S, K, 4, 7, 8)[0, :, 0, 0, :].max(0)
    miss_t = [m for m in range(8) if np.all(tau[[k for k in range(K) if k not in missing], m] == 0)]
    assert int(zc.sum()) == len(miss_t) * int(paper["l224_spatial_dim"])


def test_sref_equals_rms_constant_response():
    """Eq. 17: with a hat range covering every source time, A applied to the
    constant history x = 1 gives sum_e w_e in every frame (partition of unity),
    whose RMS over direct data is s_ref."""
    w = I.Workload("cover", I.Geometry(0.5, 50.0, 24), I.SourceGrid(5, 8),
                   I.TimeGrid(6, 1.0, 40, t_end=20.0), supersample=2)
    tab = O.build_table(w, I.screen_samples(w))
    d = tab.select((0,))
    y = O.apply_A(w, d, np.ones((w.grid.n_nodes, w.time.n_hats)), 1.0)
    assert O.s_ref(tab) == pytest.approx(np.sqrt(np.mean(y ** 2)), rel=1e-12)


def test_probe_normalisation_and_support(paper):
    """Eq. 11: N_h makes q_a unit-norm over the annulus x time (quadrature);
    Sec. 3.3: |t + a| <= 3h holds 1 - erfc(3) of the squared energy."""
    w = I.kerr256()
    Nh = O.probe_norm_const(w)
    h = paper["probe_h"]
    g = w.grid
    radial, _ = integrate.quad(lambda r: r, g.r_in, g.r_out)
    temporal, _ = integrate.quad(lambda t: math.exp(-t * t / h ** 2), -60, 60)
    assert 2 * math.pi * radial * temporal / Nh ** 2 == pytest.approx(1.0, rel=1e-12)
    inside, _ = integrate.quad(lambda t: math.exp(-t * t / h ** 2), -3 * h, 3 * h)
    assert inside / temporal == pytest.approx(paper["probe_3h_energy"], abs=1e-6)
    assert inside / temporal == pytest.approx(1 - special.erfc(3), rel=1e-12)


def test_probe_info_brute_force(tiny_kerr):
    """I(a) from the C loops == a numpy evaluation of Eq. 29 term by term."""
    w, tab = tiny_kerr
    ages = np.array([0.0, 4.0, 12.0])
    got = O.probe_info(w, tab, 7.0, ages)
    Nh = O.probe_norm_const(w)
    to = w.time.frame_times()
    ref = []
    for a in ages:
        acc = 0.0
        for row in range(tab.n_rows):
            e = slice(tab.row_ptr[row], tab.row_ptr[row + 1])
            v = np.sum(tab.weight[e][:, None] / Nh *
                       np.exp(-(to[None, :] - tab.delay[e][:, None] + a) ** 2 / 18.0), axis=0)
            acc += np.sum(v * v)
        ref.append(49.0 * acc)
    assert np.allclose(got, ref, rtol=1e-12)


def test_reach_anchor_and_jold_hand_cases(schw):
    w, tab = schw
    ages = O.AGES
    info = np.zeros(ages.size)
    info[:6] = 2.0  # ages 0..20 pass
    info[8] = 5.0  # isolated passing age 32
    fp = O.footprints(w, tab, (0,))
    r = O.reach(w, tab, info, (0,))
    # anchor: youngest age with [-a-9, -a+9] inside W_0
    lo, hi = fp[0]
    exp_anchor = next(a for a in ages if -a - 9 >= lo and -a + 9 <= hi)
    assert r.anchor == exp_anchor
    if exp_anchor <= 20:
        assert r.L_anchor == 20.0 - exp_anchor
    assert r.T_reach == 32.0
    # ages > 10 that carry information: 12, 16, 20 (I = 2) and 32 (I = 5)
    assert O.j_old(info, 10.0) == pytest.approx(4.0 * (3 * math.log(3.0) + math.log(6.0)))
    # strict '>': the age 12 itself is excluded when A_0 = 12
    assert O.j_old(info, 12.0) == pytest.approx(4.0 * (2 * math.log(3.0) + math.log(6.0)))


def test_a0999_brute_force(schw):
    w, tab = schw
    d = tab.select((0,))
    to = w.time.frame_times()
    samples = sorted((de - t, tau) for de, tau in zip(d.delay, d.throughput) for t in to)
    tot = sum(tau for _, tau in samples)
    acc = 0.0
    for age, tau in samples:
        acc += tau
        if acc >= 0.999 * tot:
            break
    assert O.a0999(w, tab) == pytest.approx(age, abs=1e-12)


def test_class_structure():
    """S224 (Eq. 8): the radial B-splines form a partition of unity, so the
    constant reference source j_ref = 1 lies in the class (Sec. 3.5); L224
    temporal hats also sum to one on the window."""
    w = I.schw32()
    Q = O.synth_class(w, "S224").reshape(w.grid.n_nodes, w.time.n_hats, 4, 7, 8)
    const = Q[:, :, :, 0, 0].sum(axis=2)
    assert np.allclose(const, 1.0, atol=1e-14)
    QL = O.synth_class(w, "L224").reshape(w.grid.n_nodes, w.time.n_hats, 4, 7, 8)
    assert np.allclose(QL[:, :, :, 0, :].sum(axis=(2, 3)), 1.0, atol=1e-14)
    assert np.linalg.matrix_rank(O.synth_class(w, "S224")) == min(224, w.n_dof)


def test_operational_rank_eigh_vs_svd(schw):
    """Rank from the Gram spectrum (eigh) equals the count from an SVD of P."""
    w, tab = schw
    scl = O.scale(tab)
    P = O.restricted_response(w, tab, O.synth_class(w, "S224"), scl)
    spec = O.operational_rank(O.gram(P))
    sv = np.linalg.svd(P, compute_uv=False)
    assert spec.rank == int(np.count_nonzero(sv >= 1.0))
    k = min(20, sv.size)
    assert np.allclose(spec.sigma[:k], sv[:k], rtol=1e-8)


def test_ridge_cg_against_dense_solve(tiny_kerr):
    w, tab = tiny_kerr
    scl = 0.8
    D = O.dense_A(w, tab, scl)
    xt = I.history_batch(w, [5])
    data = O.apply_A(w, tab, xt, scl) + 0.1 * I.noise((tab.n_rows, w.time.n_frames, 1), 6)
    x, it = O.ridge_cg(w, tab, scl, data, lam=0.3, tol=1e-13)
    ref = np.linalg.solve(D.T @ D + 0.3 * np.eye(D.shape[1]), D.T @ data.reshape(-1))
    assert np.allclose(x.reshape(-1), ref, rtol=1e-9, atol=1e-11 * np.abs(ref).max())
    res = D.T @ (D @ x.reshape(-1)) + 0.3 * x.reshape(-1) - D.T @ data.reshape(-1)
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(D.T @ data.reshape(-1))


def test_tsvd_against_svd_of_dense_response(tiny_kerr):
    """TSVD in a class (Sec. 9): the oracle's route (eigenpairs of the Gram,
    matrix-free A^T d) against the SVD of the dense P = A Q assembled per ray,
    x = Q sum_{i<r} v_i (u_i . d) / s_i; the operational rank is the count of
    singular values at or above rho."""
    w, tab = tiny_kerr
    scl = 0.8
    Q = O.synth_class(w, "S224")
    P = O.dense_A(w, tab, scl) @ Q
    U, s, Vt = np.linalg.svd(P, full_matrices=False)
    data = O.apply_A(w, tab, I.history_batch(w, [2, 9]), scl) \
        + 0.05 * I.noise((tab.n_rows, w.time.n_frames, 2), 4)
    dv = data.reshape(-1, 2)
    rho = 0.5 * (s[5] + s[6])  # a threshold well away from every singular value
    r_want = int(np.count_nonzero(s >= rho))
    assert r_want == 6
    x, r = O.tsvd_in_class(w, tab, scl, Q, data, None, rho=rho)
    assert r == r_want
    ref = Q @ (Vt[:r].T @ ((U[:, :r].T @ dv) / s[:r, None]))
    np.testing.assert_allclose(x.reshape(-1, 2), ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    # data inside the retained span is recovered exactly: d = P v_0 -> Q v_0
    d0 = (P @ Vt[0]).reshape(tab.n_rows, w.time.n_frames, 1)
    x0, _ = O.tsvd_in_class(w, tab, scl, Q, d0, 3)
    np.testing.assert_allclose(x0.reshape(-1), Q @ Vt[0], rtol=0, atol=1e-9 * np.abs(Q @ Vt[0]).max())


def test_results_do_not_depend_on_the_thread_count(tiny_kerr):
    """The C oracle's OpenMP loops write disjoint outputs: A, A^T and the probe
    information are bitwise the same on one thread and on all of them."""
    w, tab = tiny_kerr
    x = I.history_batch(w, [3, 4])
    y = O.apply_A(w, tab, x, 0.7)
    runs = []
    n_all = O.max_threads()
    try:
        for n in (1, n_all):
            O.set_threads(n)
            assert O.max_threads() == n
            runs.append((O.apply_A(w, tab, x, 0.7), O.apply_AT(w, tab, y, 0.7),
                         O.probe_info(w, tab, 0.7)))
    finally:
        O.set_threads(n_all)
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)
