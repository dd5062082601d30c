"""Pins of the oracle's ray tracing against closed forms and brute force.

Sec. 5 of the paper: the exact Schwarzschild branch reproduces r_+ = 2M,
r_ph = 3M, b_c = 3 sqrt(3) M; Kerr maps for n = 0, 1, 2 (Sec. 6.1, Eq. 38).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2609_05528_b300 import inputs as I


def test_carlson_rf_closed_forms():
    L = O.lib()
    for x in (0.3, 1.0, 7.5):
        assert L.orc_carlson_rf(x, x, x) == pytest.approx(1.0 / math.sqrt(x), rel=1e-14)
    assert L.orc_carlson_rf(0.0, 1.0, 1.0) == pytest.approx(math.pi / 2, rel=1e-14)
    # R_F(0, 1, 2) = Gamma(1/4)^2 / (4 sqrt(2 pi))  (lemniscate case)
    ref = math.gamma(0.25) ** 2 / (4.0 * math.sqrt(2.0 * math.pi))
    assert L.orc_carlson_rf(0.0, 1.0, 2.0) == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("b", [5.2, 5.5, 8.0, 40.0])
def test_orbit_integral_matches_quadrature(b):
    """psi(u) = int_0^u du / sqrt(1/b^2 - u^2 + 2u^3) in closed form (R_F) vs
    scipy's adaptive quadrature of the same integrand."""
    L = O.lib()
    ut = L.orc_schw_turning_u(b)
    assert 1.0 / b ** 2 - ut ** 2 + 2 * ut ** 3 == pytest.approx(0.0, abs=1e-15)
    for frac in (0.05, 0.5, 0.9, 0.999):
        u = frac * ut
        ref, _ = integrate.quad(lambda v: 1.0 / math.sqrt(1.0 / b ** 2 - v * v + 2 * v ** 3), 0.0, u,
                                epsabs=1e-14, epsrel=1e-13, limit=200)
        assert L.orc_schw_psi(b, u) == pytest.approx(ref, rel=1e-10)


def test_critical_impact_parameter_and_photon_sphere(paper):
    """Bisection on capture vs escape with the Kerr integrator at a = 0 finds
    b_c = 3 sqrt 3; near-critical scattered rays turn at r -> r_ph = 3."""
    lo, hi = 5.0, 5.4
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        fate, _ = O.kerr_fate(0.0, math.radians(30.0), mid, 0.0)
        if fate < 0:
            lo = mid
        else:
            hi = mid
    assert 0.5 * (lo + hi) == pytest.approx(paper["schw_b_c"], abs=1e-8)
    fate, rmin = O.kerr_fate(0.0, math.radians(30.0), paper["schw_b_c"] + 1e-9, 0.0)
    assert fate == 1
    assert rmin == pytest.approx(paper["schw_r_ph"], abs=1e-3)
    assert O.horizon(0.0) == paper["schw_r_plus"]


def test_kerr_integrator_at_a0_matches_exact_schwarzschild():
    w = I.schw32()
    s = I.screen_samples(w)
    ts = O.trace(0.0, w.geometry.incl, s.alpha, s.beta, method="schw")
    tk = O.trace(0.0, w.geometry.incl, s.alpha, s.beta, method="kerr")
    v1 = ts.found & (ts.r >= 3) & (ts.r <= 11)
    v2 = tk.found & (tk.r >= 3) & (tk.r <= 11)
    assert np.array_equal(v1, v2)
    assert v1[:, 0].sum() > 500 and v1[:, 1].sum() > 10
    m = v1
    assert np.max(np.abs(ts.r - tk.r)[m]) < 1e-9
    assert np.max(np.abs(np.angle(np.exp(1j * (ts.phi - tk.phi))))[m]) < 2e-9
    assert np.max(np.abs(ts.T - tk.T)[m]) < 2e-9
    assert np.array_equal(ts.sr[m], tk.sr[m])


def test_schwarzschild_order_structure():
    """Radial screen scan (Schwarzschild, near face-on): the width of the n=2
    band over r in [3, 11] is e^{-pi} of the n=1 band (Lyapunov exponent pi),
    and the delay of the same source ring grows by pi sqrt(27) per order for
    n >= 1 (half an orbit of the photon sphere)."""
    incl = math.radians(1.0)
    b = np.linspace(5.19, 7.0, 6001)
    tr = O.trace(0.0, incl, b, np.zeros_like(b), n_orders=4, r_esc=1e6, method="schw")
    widths = []
    for n in (1, 2):
        ok = tr.found[:, n] & (tr.r[:, n] >= 3) & (tr.r[:, n] <= 11)
        widths.append(b[ok].max() - b[ok].min())
    assert widths[1] / widths[0] == pytest.approx(math.exp(-math.pi), rel=0.25)
    half_orbit = math.pi * math.sqrt(27.0)
    for rs in (4.0, 6.0, 9.0):
        Tn = []
        for n in (1, 2, 3):
            ok = tr.found[:, n]
            rr, TT = tr.r[ok, n], tr.T[ok, n]
            # r decreases with b along each order's band; interpolate T at r = rs
            o = np.argsort(rr)
            Tn.append(np.interp(rs, rr[o], TT[o]))
        assert Tn[1] - Tn[0] == pytest.approx(half_orbit, rel=0.10)
        assert Tn[2] - Tn[0] == pytest.approx(2 * half_orbit, rel=0.10)


def _bardeen_curve(a, incl, n=20001):
    rm = 2.0 * (1.0 + math.cos(2.0 / 3.0 * math.acos(-a)))
    rp = 2.0 * (1.0 + math.cos(2.0 / 3.0 * math.acos(a)))
    r = np.linspace(rm, rp, n)
    D = r * r - 2 * r + a * a
    lam = a + r / a * (r - 2 * D / (r - 1))
    eta = r ** 3 / a ** 2 * (4 * D / (r - 1) ** 2 - r)
    al = -lam / math.sin(incl)
    b2 = eta + a * a * math.cos(incl) ** 2 - lam ** 2 / math.tan(incl) ** 2
    ok = b2 >= 0
    al, be = al[ok], np.sqrt(b2[ok])
    return np.concatenate([al, al]), np.concatenate([be, -be])


@pytest.mark.parametrize("a,incl_deg", [(0.5, 50.0), (0.94, 75.0)])
def test_kerr_n2_images_hug_bardeen_curve(a, incl_deg):
    """Higher-order images approach the critical curve (Bardeen 1973 closed
    form): every n=2 ray lies within 0.3 M of it and the mean n=2 offset is
    about e^{-pi} of the mean n=1 offset."""
    w = I.small_kerr(spin=a, incl_deg=incl_deg, nx=96, ss=2)
    s = I.screen_samples(w)
    tab = O.build_table(w, s)
    ca, cb = _bardeen_curve(a, math.radians(incl_deg))
    dist = {}
    for n in (1, 2):
        idx = tab.sample[tab.order == n]
        d = np.min(np.hypot(s.alpha[idx, None] - ca[None, :], s.beta[idx, None] - cb[None, :]), axis=1)
        dist[n] = d
    assert dist[2].max() < 0.3
    assert 0.01 < dist[2].mean() / dist[1].mean() < 0.25


def test_delay_increment_matches_eq38(paper):
    """Eq. 38 (a = 0.5, i = 50 deg): the n = 1 -> 2 delay ranges are offset
    by 16.1 M (minima) and 16.8 M (maxima), i.e. about pi sqrt(27)."""
    w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=96, ss=2)
    tab = O.build_table(w, I.screen_samples(w))
    d1 = tab.delay[tab.order == 1]
    d2 = tab.delay[tab.order == 2]
    inc_min = d2.min() - d1.min()
    inc_max = d2.max() - d1.max()
    paper_inc = 0.5 * ((paper["eq38_n2_min"] - paper["eq38_n1_min"]) +
                       (paper["eq38_n2_max"] - paper["eq38_n1_max"]))
    assert inc_min == pytest.approx(paper_inc, rel=0.12)
    assert inc_max == pytest.approx(paper_inc, rel=0.12)


def test_redshift_closed_forms():
    """Schwarzschild Keplerian emitter seen along the axis (lambda = 0):
    g = sqrt(1 - 3/r).  ISCO E, L = sqrt(8/9), 2 sqrt(3) at r = 6.  The
    plunging branch joins the circular branch continuously at the ISCO."""
    r = np.array([6.0, 7.5, 11.0])
    g = O.redshift(0.0, r, 0.0, 20.0, 1.0)
    assert np.allclose(g, np.sqrt(1 - 3 / r), rtol=1e-14)
    assert O.isco(0.0) == pytest.approx(6.0, rel=1e-14)
    E, L = O.circular_EL(0.0, 6.0)
    assert E == pytest.approx(math.sqrt(8 / 9), rel=1e-14)
    assert L == pytest.approx(2 * math.sqrt(3), rel=1e-14)
    for a in (0.0, 0.5, 0.94):
        rI = O.isco(a)
        for lam, eta, sr in ((2.0, 15.0, 1.0), (-3.0, 20.0, -1.0)):
            g_out = O.redshift(a, np.array([rI * (1 + 1e-9)]), lam, eta, sr)[0]
            g_in = O.redshift(a, np.array([rI * (1 - 1e-9)]), lam, eta, sr)[0]
            assert g_in == pytest.approx(g_out, rel=1e-4)


def test_isco_closed_forms_and_marginal_stability():
    """The ISCO that sets the circular/plunging branch (Sec. 5) against what
    fixes it without the Bardeen-Press-Teukolsky closed form: the extreme
    cases r = 1 (a = 1, prograde) and r = 9 (a = 1, retrograde), r = 6 at
    a = 0, the tabulated 4.233 (a = 0.5) and 2.3209 (a = 0.9), and the
    marginal-stability definition: the ISCO is where the circular orbit's
    specific energy E(r) has its minimum, found here by brute-force search on
    circular_EL (which the Schwarzschild values above pin independently)."""
    from scipy import optimize
    assert O.isco(1.0) == pytest.approx(1.0, abs=1e-12)
    assert O.isco(-1.0) == pytest.approx(9.0, abs=1e-12)
    assert O.isco(0.0) == pytest.approx(6.0, abs=1e-12)
    assert O.isco(0.5) == pytest.approx(4.233, abs=5e-4)
    assert O.isco(0.9) == pytest.approx(2.3209, abs=5e-4)
    for a in (0.3, 0.5, 0.75, 0.94, -0.5):
        rI = O.isco(a)
        # coarse scan for the bracket, then a bounded scalar minimisation
        rs = np.linspace(rI * 0.6, rI * 1.8, 4001)
        rs = rs[rs ** 1.5 - 3.0 * np.sqrt(rs) + 2.0 * a > 1e-9]
        E = O.circular_EL(a, rs)[0]
        i = int(np.argmin(E))
        res = optimize.minimize_scalar(lambda r: float(O.circular_EL(a, r)[0]),
                                       bounds=(rs[max(i - 2, 0)], rs[min(i + 2, rs.size - 1)]),
                                       method="bounded", options={"xatol": 1e-10})
        assert res.x == pytest.approx(rI, rel=2e-6), a
