"""Pins of the oracle's order mixing (Sec. 3.1 Eq. 4): the unresolved image
and the total-flux readout as whitened linear collapses of the order-resolved
data, with the noise propagated through the same map."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import inputs as I


class _Rows:
    """The two row fields the mixer reads."""

    def __init__(self, order, pixel):
        self.row_order = np.asarray(order, np.int8)
        self.row_pixel = np.asarray(pixel, np.int32)


def test_hand_worked_example():
    """Rows (order, pixel) = (0, 5), (0, 7), (1, 5), (1, 9), (2, 5) with data
    1, 2, 3, 4, 5 (one frame, one history).  Unresolved: pixel 5 collects
    orders 0, 1, 2 -> (1 + 3 + 5) / sqrt(3); pixel 7 -> 2 / 1; pixel 9 -> 4 / 1.
    Total flux: (1 + 2 + 3 + 4 + 5) / sqrt(5).  Direct arm only: the two
    direct rows unchanged."""
    t = _Rows([0, 0, 1, 1, 2], [5, 7, 5, 9, 5])
    y = np.array([1.0, 2.0, 3.0, 4.0, 5.0]).reshape(5, 1, 1)
    u = O.mix_rows(t, y, O.MIX_UNRESOLVED)
    assert u.shape == (3, 1, 1)
    np.testing.assert_allclose(u.ravel(), [9.0 / math.sqrt(3.0), 2.0, 4.0], rtol=1e-15)
    f = O.mix_rows(t, y, O.MIX_TOTAL_FLUX)
    np.testing.assert_allclose(f.ravel(), [15.0 / math.sqrt(5.0)], rtol=1e-15)
    d = O.mix_rows(t, y[:2], O.MIX_UNRESOLVED, orders=(0,))
    np.testing.assert_allclose(d.ravel(), [1.0, 2.0], rtol=0)
    # adjoint: each row receives its pixel's value over sqrt(its row count)
    back = O.mix_rows_T(t, np.array([1.0, 1.0, 1.0]).reshape(3, 1, 1), O.MIX_UNRESOLVED)
    s3 = 1.0 / math.sqrt(3.0)
    np.testing.assert_allclose(back.ravel(), [s3, 1.0, s3, 1.0, s3], rtol=1e-15)


@pytest.fixture(scope="module")
def schw():
    w = I.schw32()
    return w, O.build_table(w, I.screen_samples(w))


@pytest.mark.parametrize("mode", [O.MIX_UNRESOLVED, O.MIX_TOTAL_FLUX])
@pytest.mark.parametrize("orders", [(0, 1, 2), (0, 1), (0,)])
def test_mixed_noise_is_white(schw, mode, orders):
    """W W^T = I: whitened rows stay unit-variance after the collapse, so no
    arm gets an independent noise level (Sec. 4.2)."""
    _, tab = schw
    W = O.mixer(tab, mode, orders)
    WW = (W @ W.T).toarray()
    np.testing.assert_allclose(WW, np.eye(W.shape[0]), atol=1e-15)


def test_direct_arm_unresolved_is_identity(schw):
    """With the direct order alone every pixel has one row: no collapse."""
    _, tab = schw
    W = O.mixer(tab, O.MIX_UNRESOLVED, (0,)).toarray()
    assert W.shape[0] == W.shape[1] == tab.rows_of_order(0)
    np.testing.assert_array_equal(W, np.eye(W.shape[0]))


def test_unresolved_brute_force(schw):
    """Per pixel, loop over the rows of every order with that pixel, add them
    and divide by the square root of their count; compare with W y."""
    w, tab = schw
    rng = np.random.default_rng(3)
    y = rng.standard_normal((tab.n_rows, w.time.n_frames, 2))
    got = O.mix_rows(tab, y, O.MIX_UNRESOLVED)
    pixels = sorted(set(int(p) for p in tab.row_pixel))
    assert got.shape[0] == len(pixels)
    for i, p in enumerate(pixels):
        rows = [r for r in range(tab.n_rows) if int(tab.row_pixel[r]) == p]
        want = sum(y[r] for r in rows) / math.sqrt(len(rows))
        np.testing.assert_allclose(got[i], want, rtol=1e-13, atol=1e-13)
    assert any(sum(1 for r in range(tab.n_rows) if int(tab.row_pixel[r]) == p) > 1 for p in pixels)


def test_total_flux_of_constant_rows(schw):
    """Constant data c on R rows: the total-flux readout is c R / sqrt(R)."""
    w, tab = schw
    y = np.full((tab.n_rows, w.time.n_frames, 1), 2.5)
    f = O.mix_rows(tab, y, O.MIX_TOTAL_FLUX)
    np.testing.assert_allclose(f, 2.5 * math.sqrt(tab.n_rows), rtol=1e-14)


@pytest.mark.parametrize("mode", [O.MIX_UNRESOLVED, O.MIX_TOTAL_FLUX])
def test_collapse_never_adds_information(schw, mode):
    """P = W^T W is an orthogonal projector, so the collapsed Gram
    B^T P B is below the resolved Gram B^T B: every eigenvalue is at most the
    resolved one (Weyl), and the total-flux Gram has rank at most T."""
    w, tab = schw
    scl = O.scale(tab)
    Q = O.synth_class(w, "S224")
    P = O.restricted_response(w, tab, Q, scl)  # [rows * T, d]
    T = w.time.n_frames
    d = P.shape[1]
    W = O.mixer(tab, mode)
    Pl = O.mix_rows(tab, P.reshape(tab.n_rows, T, d), mode).reshape(-1, d)
    lr = np.linalg.eigvalsh(P.T @ P)
    ll = np.linalg.eigvalsh(Pl.T @ Pl)
    assert np.all(ll <= lr + 1e-9 * lr.max())
    PP = (W.T @ W).toarray()
    np.testing.assert_allclose(PP @ PP, PP, atol=1e-14)
    if mode == O.MIX_TOTAL_FLUX:
        assert np.sum(ll > 1e-9 * ll.max()) <= T


def test_mixed_probe_identity_arm_matches_c_probe(schw):
    """Direct arm, unresolved collapse = identity: the numpy mixed probe
    information equals the C oracle's probe information on the direct rows."""
    w, tab = schw
    scl = O.scale(tab)
    got = O.mix_probe_info(w, tab, scl, O.MIX_UNRESOLVED, (0,))
    want = O.probe_info(w, tab.select((0,)), scl)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)
    assert np.max(want) > 1.0


@pytest.mark.parametrize("mode", [O.MIX_UNRESOLVED, O.MIX_TOTAL_FLUX])
def test_mixed_probe_below_resolved(schw, mode):
    """W^T W is a projector, so the collapsed probe information never exceeds
    the resolved one (C oracle), age by age; and it is strictly below it at
    some age (the orders do not all coincide)."""
    w, tab = schw
    scl = O.scale(tab)
    got = O.mix_probe_info(w, tab, scl, mode)
    res = O.probe_info(w, tab, scl)
    assert np.all(got <= res * (1 + 1e-12))
    assert np.any(got < 0.999 * res)


def test_pairing_destroyed_keeps_marginals(schw):
    """The pairing-destroyed control's delays: each order keeps its multiset of
    delays, rays move only within their order, the pairing changes, and the
    construction is a function of the keys alone."""
    w, tab = schw
    keys = I.uniforms(11, tab.n_rays)
    pd = O.pairing_destroyed(tab, keys)
    for n in range(3):
        m = tab.order == n
        np.testing.assert_array_equal(np.sort(pd.delay[m]), np.sort(tab.delay[m]))
    assert np.count_nonzero(pd.delay != tab.delay) > tab.n_rays // 2
    for k in ("order", "pixel", "r", "phi", "weight", "throughput"):
        np.testing.assert_array_equal(getattr(pd, k), getattr(tab, k))
    np.testing.assert_array_equal(O.pairing_destroyed(tab, keys).delay, pd.delay)
    # with keys that sort like the indices the permutation is the identity
    ident = O.pairing_destroyed(tab, np.arange(tab.n_rays, dtype=np.float64))
    np.testing.assert_array_equal(ident.delay, tab.delay)


def test_pairing_destroyed_hand_case():
    """Order 0 rays 0, 2, 3 with keys 0.7, 0.1, 0.4 sort by key as 2, 3, 0:
    ray 0 takes ray 2's delay, ray 2 ray 3's, ray 3 ray 0's.  The single
    order-1 ray keeps its delay."""
    t = _hand_table([0, 1, 0, 0], [10.0, 20.0, 30.0, 40.0])
    got = O.pairing_destroyed(t, [0.7, 0.9, 0.1, 0.4])
    assert got.delay.tolist() == [30.0, 20.0, 40.0, 10.0]


def test_local_direction_norms_by_2d_quadrature(schw):
    """N_{h,l}^2 / (h sqrt(pi)) equals the area integral of psi_l^2 over the
    annulus, computed here as one 2D integral in (r, phi)."""
    from scipy import integrate
    w, _ = schw
    g = w.grid
    N = O.local_direction_norms(w)
    for l in (0, 3, 9, 20, 27):
        f = lambda ph, r, l=l: O.local_direction_values(w, np.array([r]), np.array([ph]))[0, l] ** 2 * r
        area, _ = integrate.dblquad(f, g.r_in, g.r_out, 0.0, 2 * math.pi, epsabs=0, epsrel=1e-10)
        assert abs(N[l] ** 2 / (O.PROBE_H * math.sqrt(math.pi)) / area - 1.0) < 1e-8


def test_local_directions_rebuild_the_scalar_probe(schw):
    """The radial Bernstein polynomials sum to one, so the four l = 0
    directions, each times N_{h,(i,0)} / N_h, add up to the scalar probe q_a:
    their responses rebuild the scalar probe information (C oracle)."""
    w, tab = schw
    scl = O.scale(tab)
    N = O.local_direction_norms(w)
    Nh = O.probe_norm_const(w)
    ages = [0.0, 8.0, 24.0]
    for a, want in zip(ages, O.probe_info(w, tab, scl, ages)):
        Y = O.local_probe_responses(w, tab, a)
        ys = sum(Y[7 * i] * N[7 * i] / Nh for i in range(4))
        assert abs(scl * scl * np.sum(ys ** 2) / want - 1.0) < 1e-12
    loc = O.local_probe_info(w, tab, scl, ages=ages)
    assert loc.shape == (3, 28) and np.all(loc >= 0)


def test_local_reach_hand_cases():
    """The deepest age with any direction at or above rho^2: the passing
    direction may change with age; an age where none passes between two that
    do does not cut the reach (it is the last passing age, not a run)."""
    ages = [0.0, 4.0, 8.0, 12.0]
    info = np.array([[2.0, 0.0], [0.0, 1.0], [0.5, 0.2], [0.0, 0.0]])
    assert O.local_reach(info, 1.0, ages) == 4.0
    info[2, 0] = 4.0
    assert O.local_reach(info, 2.0, ages) == 8.0
    assert O.local_reach(info, 2.01, ages) is None  # 4 < 2.01^2: nothing passes
    assert O.local_reach(info, 1.4, ages) == 8.0    # age 0 (2 >= 1.96) and age 8
    assert O.local_reach(np.zeros((4, 2)), 1.0, ages) is None
    gap = np.array([[1.0], [0.0], [1.0], [0.0]])
    assert O.local_reach(gap, 1.0, ages) == 8.0


def _hand_table(order, delay):
    order = np.asarray(order, np.int8)
    n = order.size
    delay = np.asarray(delay, np.float64)
    r = 3.0 + np.arange(n, dtype=np.float64)
    phi = 0.1 * np.arange(n, dtype=np.float64)
    one = np.ones(n)
    return O.Table(order, np.arange(n, dtype=np.int32), r, phi, delay, one, one.copy(),
                   np.arange(n + 1, dtype=np.int64), order.copy(), np.arange(n, dtype=np.int32),
                   np.arange(n, dtype=np.int64))


def test_direct_quantile_partner_hand_case():
    """Direct ranking by delay: rays 1, 3, 0, 2.  Order 1 (two rays): ray 5
    (k = 0) -> rank floor(0.5 * 4 / 2) = 1 -> ray 3; ray 4 (k = 1) -> rank 3
    -> ray 2.  Order 2 (one ray): rank floor(0.5 * 4) = 2 -> ray 0.  Direct
    rays map to themselves.  The arms then move source points (delay-only)
    or delays (spatial-only) of the ring rays from these partners."""
    order = [0, 0, 0, 0, 1, 1, 2]
    delay = [3.0, 1.0, 4.0, 2.0, 9.0, 7.0, 20.0]
    t = _hand_table(order, delay)
    assert O.quantile_partner(t).tolist() == [0, 1, 2, 3, 2, 3, 0]
    do = O.delay_only(t)
    assert do.r.tolist() == [3.0, 4.0, 5.0, 6.0, 5.0, 6.0, 3.0]
    assert do.delay.tolist() == delay
    so = O.spatial_only(t)
    assert so.delay.tolist() == [3.0, 1.0, 4.0, 2.0, 4.0, 2.0, 3.0]
    assert so.r.tolist() == t.r.tolist()
    # ties in delay are broken by ray index on both rankings
    t2 = _hand_table([0, 0, 1, 1], [5.0, 5.0, 8.0, 8.0])
    assert O.quantile_partner(t2).tolist() == [0, 1, 0, 1]


def test_spatial_only_keeps_direct_old_epoch_blindness(schw):
    """Spatial-only arm: the rings keep source points, weights and rows, and
    their delays, rank for rank, become direct delays.  Every order's
    footprint then lies inside the direct one, so Theorem 4.1's blind columns
    of the direct image (hats whose support misses W_0) stay exactly zero in
    the whole stack, while the true resolved stack sees some of them."""
    w, tab = schw
    so = O.spatial_only(tab)
    ring = tab.order > 0
    for k in ("order", "pixel", "r", "phi", "weight", "throughput"):
        np.testing.assert_array_equal(getattr(so, k), getattr(tab, k))
    np.testing.assert_array_equal(so.delay[~ring], tab.delay[~ring])
    assert np.all(np.isin(so.delay[ring], tab.delay[~ring]))
    for n in (1, 2):
        m = np.nonzero(tab.order == n)[0]
        if m.size:
            assert np.all(np.diff(so.delay[m[np.argsort(tab.delay[m], kind="stable")]]) >= 0)
    scl = O.scale(tab)
    zero = lambda t: np.all(O.dense_A(w, t, scl) == 0.0, axis=0)  # noqa: E731
    zs = zero(so)
    zr = zero(tab)
    (lo, hi), = O.footprints(w, tab, (0,))
    tk = w.time.hat_times()
    miss = (tk + w.time.hat_step <= lo) | (tk - w.time.hat_step >= hi)  # hat misses W_0
    blind = np.tile(miss, w.grid.n_nodes)  # columns s * K + k
    assert blind.sum() > 0
    assert np.all(zs[blind]) and not np.all(zr[blind])


@pytest.mark.parametrize("case", ["schw32", "small_kerr"])
def test_delay_only_and_spatial_only_reach(case):
    """The scalar probe (Eq. 10) is the same at every source point of the
    annulus, so the delay-only arm (ring source points moved, delays kept)
    has the resolved stack's probe information, reach and J_old exactly, as
    the paper's Sec. 6.4 reports equal medians for the two.  The
    spatial-only arm stays near the direct image (at most 5% more J_old,
    never the resolved value)."""
    w = I.schw32() if case == "schw32" else I.small_kerr(
        spin=0.5, incl_deg=50.0, nx=64, n_r=8, n_phi=16, n_frames=128, n_hats=32, ss=2)
    tab = O.build_table(w, I.screen_samples(w))
    scl = O.scale(tab)
    a0 = O.a0999(w, tab)
    td = O.delay_only(tab)
    ring = tab.order > 0
    for k in ("order", "pixel", "delay", "weight", "throughput"):
        np.testing.assert_array_equal(getattr(td, k), getattr(tab, k))
    direct_pts = set(zip(tab.r[~ring].tolist(), tab.phi[~ring].tolist()))
    assert all(p in direct_pts for p in zip(td.r[ring].tolist(), td.phi[ring].tolist()))
    ts = O.spatial_only(tab)
    assert O.scale(td) == scl and O.scale(ts) == scl  # direct rays untouched
    info = {name: O.probe_info(w, t.select(orders), scl)
            for name, t, orders in (("direct", tab, (0,)), ("resolved", tab, (0, 1, 2)),
                                    ("delay_only", td, (0, 1, 2)),
                                    ("spatial_only", ts, (0, 1, 2)))}
    np.testing.assert_allclose(info["delay_only"], info["resolved"], rtol=1e-13, atol=0)
    J = {k: O.j_old(v, a0) for k, v in info.items()}
    assert J["direct"] <= J["spatial_only"] <= 1.05 * J["direct"] < J["resolved"]
    r_res = O.reach(w, tab, info["resolved"], (0, 1, 2))
    r_do = O.reach(w, td, info["delay_only"], (0, 1, 2))
    assert r_do.L_anchor == r_res.L_anchor and r_res.L_anchor > 0
    # the delay-only stack touches only nodes the direct image touches
    nz = lambda t: np.any(O.dense_A(w, t, scl) != 0.0, axis=0).reshape(  # noqa: E731
        w.grid.n_nodes, w.time.n_hats).any(axis=1)
    if case == "schw32":
        assert not np.any(nz(td) & ~nz(tab.select((0,))))


@pytest.mark.parametrize("mode", [O.MIX_UNRESOLVED, O.MIX_TOTAL_FLUX])
def test_mixed_arm_reach_never_exceeds_resolved(schw, mode):
    """The mixed arms use the resolved footprints (the union of the summed
    orders') and the direct A_{0,0.999}; their probe information is below the
    resolved one age by age, so their J_old is too, and their passing ages
    are a subset of the resolved ones."""
    w, tab = schw
    scl = O.scale(tab)
    res = O.probe_info(w, tab, scl)
    mix = O.mix_probe_info(w, tab, scl, mode)
    a0 = O.a0999(w, tab)
    assert O.j_old(mix, a0) <= O.j_old(res, a0) * (1 + 1e-12)
    r_res = O.reach(w, tab, res, (0, 1, 2))
    r_mix = O.reach(w, tab, mix, (0, 1, 2))
    assert not np.any(r_mix.passing & ~r_res.passing)
    assert r_mix.anchor == r_res.anchor  # the anchor depends on the footprints only
    assert r_mix.L_anchor <= r_res.L_anchor
