/*
 * rtt_oracle.c -- plain, slow, FP64 CPU oracle for the multi-order
 * retarded-time imaging operator (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, the smoke check and the CPU-baseline leg of bench.py may load
 * this library.  It shares no code, header or constant with the CUDA path in
 * paper_2609_05528_b300/csrc; it is compiled on its own with gcc and loaded
 * through ctypes by oracle/oracle.py.
 *
 * Contents (each function cites the passage of the paper it restates):
 *   orc_trace_kerr   null geodesics in Kerr, Mino-time Carter equations
 *                    (Sec. 3.1, Eq. 2: r_n, phi_n, Delta_n per order n;
 *                    Sec. 5: Kerr ray maps for n = 0, 1, 2).
 *   orc_trace_schw   Schwarzschild rays from the exact orbit integral
 *                    (Sec. 5: exact Schwarzschild branch, b_c = 3 sqrt(3) M).
 *   orc_apply_A      matrix-free forward action of the order-resolved stack
 *                    (Eq. 2, Eq. 3, Eq. 16, Eq. 47).
 *   orc_apply_AT     its exact transpose (Sec. 5: explicit adjoint action).
 *   orc_probe_info   age information I(a) of the scalar probe q_a
 *                    (Eq. 10, Eq. 11, Eq. 12, Eq. 29).
 *
 * Conventions (all lengths and times in units of M, M = 1):
 *   screen (alpha, beta); lambda = -alpha sin i, eta = (alpha^2-a^2) cos^2 i
 *   + beta^2.  Rays are traced backwards from an observer at infinity at
 *   inclination i and azimuth 0.  Order n is the (n+1)-th crossing of the
 *   equatorial plane.  A crossing is counted only while the ray stays outside
 *   r_+ + 0.01 (capture cushion) and before it is outgoing beyond r_esc.
 *   The regularised travel time is T = lim [t(r) - r - 2 ln r] (r -> inf)
 *   minus the emission time; delays are T minus the minimum direct T.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NSTATE 6
#define CAPTURE_CUSHION 0.01

/* ------------------------------------------------------------------------ */
/* Kerr: Mino-time equations in s = 1/r and u = cos(theta).                  */
/* (ds/dl)^2 = P(s) = R(1/s) s^4,  (du/dl)^2 = U(u)                           */
/*   R(r) = (r^2+a^2-a lam)^2 - Delta (eta + (lam-a)^2)                        */
/*   U(u) = eta - (eta + lam^2 - a^2) u^2 - a^2 u^4                           */
/* Second-order forms s'' = P'(s)/2, u'' = U'(u)/2 have no sign flips at       */
/* turning points.  phi' = -Phi, and Y is the travel time with r + 2 ln r     */
/* subtracted so that it stays finite at s = 0.                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    double a, lam, eta, K, c2, c0, uu2; /* uu2 = eta + lam^2 - a^2 */
} kerr_par;

static void kerr_setup(kerr_par* p, double a, double lam, double eta) {
    p->a = a; p->lam = lam; p->eta = eta;
    p->K = eta + (lam - a) * (lam - a);
    p->c2 = 2.0 * a * a - 2.0 * a * lam - p->K;
    p->c0 = (a * a - a * lam) * (a * a - a * lam) - a * a * p->K;
    p->uu2 = eta + lam * lam - a * a;
}

static double kerr_P(const kerr_par* p, double s) {
    return 1.0 + p->c2 * s * s + 2.0 * p->K * s * s * s + p->c0 * s * s * s * s;
}

static void kerr_rhs(const kerr_par* p, const double* y, double* dy) {
    const double a = p->a, lam = p->lam;
    const double s = y[0], vs = y[1], u = y[2], vu = y[3];
    dy[0] = vs;
    dy[1] = p->c2 * s + 3.0 * p->K * s * s + 2.0 * p->c0 * s * s * s;
    dy[2] = vu;
    dy[3] = -p->uu2 * u - 2.0 * a * a * u * u * u;
    const double dtil = 1.0 - 2.0 * s + a * a * s * s;        /* Delta / r^2 */
    const double w = 1.0 + (a * a - a * lam) * s * s;          /* (r^2+a^2-a lam)/r^2 */
    const double sin2 = 1.0 - u * u;
    const double Phi = a * w / dtil - a + lam / sin2;
    dy[4] = -Phi;
    /* dt/dl - (1+2s) sgn(vs) sqrt(P) / s^2, written without cancellation for
       the ingoing branch: see the series identity in the header comment. */
    const double Pv = kerr_P(p, s);
    const double sq = sqrt(Pv > 0.0 ? Pv : 0.0);
    const double tail = a * lam - a * a * sin2;
    if (vs >= 0.0) {
        const double q = (p->c2 + 2.0 * p->K * s + p->c0 * s * s) / (1.0 + sq);
        const double Nt = (4.0 + a * a - a * lam) - 2.0 * a * a * s +
                          a * a * (a * a - a * lam) * s * s -
                          (1.0 + 2.0 * s) * dtil * q;
        dy[5] = Nt / dtil + tail;
    } else {
        const double num = (1.0 + a * a * s * s) * w / dtil;  /* r^-2 (r^2+a^2)(..)/Delta */
        dy[5] = (num + (1.0 + 2.0 * s) * sq) / (s * s) + tail;
    }
}

/* Dormand-Prince 5(4) tableau (Dormand & Prince 1980). */
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {0.2, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
static const double DP_E[7] = {71.0 / 57600.0, 0.0, -71.0 / 16695.0, 71.0 / 1920.0,
                               -17253.0 / 339200.0, 22.0 / 525.0, -1.0 / 40.0};

/* One DP5 step of size h from y; writes y5 and returns the scaled error. */
static double dp_step(const kerr_par* p, const double* y, double h, double* y5,
                      double rtol, double atol) {
    double k[7][NSTATE], tmp[NSTATE];
    kerr_rhs(p, y, k[0]);
    for (int st = 1; st < 7; ++st) {
        for (int i = 0; i < NSTATE; ++i) {
            double acc = y[i];
            for (int j = 0; j < st; ++j) acc += h * DP_A[st][j] * k[j][i];
            tmp[i] = acc;
        }
        kerr_rhs(p, tmp, k[st]);
    }
    for (int i = 0; i < NSTATE; ++i) y5[i] = tmp[i]; /* stage 7 argument = 5th-order solution */
    double err = 0.0;
    for (int i = 0; i < NSTATE; ++i) {
        double e = 0.0;
        for (int j = 0; j < 7; ++j) e += DP_E[j] * k[j][i];
        e *= h;
        const double sc = atol + rtol * fmax(fabs(y[i]), fabs(y5[i]));
        const double r = fabs(e) / sc;
        if (r > err) err = r;
    }
    return err;
}

/* Per ray: out arrays have n_orders entries per ray (ray-major).
 * found[ray*n_orders+n] = 1 if the (n+1)-th crossing happened (any radius),
 * r, phi (in [0, 2pi)), T (regularised time), sr (forward radial direction
 * of the photon at emission, +1 outgoing / -1 ingoing).
 * Returns the number of rays that hit the step limit. */
long orc_trace_kerr(double a, double incl, long n_rays, const double* alpha,
                    const double* beta, int n_orders, double r_esc, double rtol,
                    double* r_out, double* phi_out, double* T_out, double* sr_out,
                    int8_t* found) {
    const double si = sin(incl), ci = cos(incl);
    const double r_plus = 1.0 + sqrt(1.0 - a * a);
    const double s_cap = 1.0 / (r_plus + CAPTURE_CUSHION);
    const double s_esc = 1.0 / r_esc;
    long n_bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : n_bad)
    for (long ir = 0; ir < n_rays; ++ir) {
        const double al = alpha[ir], be = beta[ir];
        kerr_par p;
        const double lam = -al * si;
        const double eta = (al * al - a * a) * ci * ci + be * be;
        kerr_setup(&p, a, lam, eta);
        for (int n = 0; n < n_orders; ++n) {
            found[ir * n_orders + n] = 0;
            r_out[ir * n_orders + n] = NAN;
            phi_out[ir * n_orders + n] = NAN;
            T_out[ir * n_orders + n] = NAN;
            sr_out[ir * n_orders + n] = 0.0;
        }
        double y[NSTATE] = {0.0, 1.0, ci, be * si, 0.0, 0.0};
        double h = 1e-4;
        int n_cross = 0;
        long steps = 0;
        const double atol = rtol;
        while (n_cross < n_orders) {
            if (++steps > 2000000) { n_bad += 1; break; }
            double y5[NSTATE];
            const double err = dp_step(&p, y, h, y5, rtol, atol);
            if (err > 1.0) {
                h *= fmax(0.2, 0.9 * pow(err, -0.2));
                continue;
            }
            /* accepted step y -> y5 over h: look for u sign change */
            if ((y[2] > 0.0 && y5[2] <= 0.0) || (y[2] < 0.0 && y5[2] >= 0.0)) {
                double hc = h * y[2] / (y[2] - y5[2]);
                double yc[NSTATE];
                for (int it = 0; it < 12; ++it) {
                    dp_step(&p, y, hc, yc, rtol, atol);
                    double dy[NSTATE];
                    kerr_rhs(&p, yc, dy);
                    const double dh = -yc[2] / dy[2];
                    hc += dh;
                    if (fabs(dh) <= 1e-16 * (fabs(hc) + 1e-300)) break;
                }
                dp_step(&p, y, hc, yc, rtol, atol);
                if (yc[0] < s_cap && yc[0] > 0.0) {
                    const double rr = 1.0 / yc[0];
                    const long o = ir * n_orders + n_cross;
                    found[o] = 1;
                    r_out[o] = rr;
                    double ph = fmod(yc[4], 2.0 * M_PI);
                    if (ph < 0.0) ph += 2.0 * M_PI;
                    phi_out[o] = ph;
                    T_out[o] = yc[5] - (rr + 2.0 * log(rr));
                    sr_out[o] = (yc[1] >= 0.0) ? 1.0 : -1.0;
                    n_cross += 1;
                } else {
                    /* crossing beyond the capture cushion or at r = inf: stop */
                    memcpy(y, y5, sizeof y);
                    break;
                }
            }
            memcpy(y, y5, sizeof y);
            if (y[0] >= s_cap) break;                   /* captured */
            if (y[1] < 0.0 && y[0] < s_esc) break;      /* escaping beyond r_esc */
            if (y[0] <= 0.0) break;                     /* reached infinity */
            h *= fmin(5.0, fmax(0.2, 0.9 * pow(fmax(err, 1e-10), -0.2)));
            if (h > 0.02) h = 0.02;
        }
    }
    return n_bad;
}

/* Fate of one ray with no crossing limit: -1 captured (reached r_+ + 0.01),
 * +1 escaped (back to infinity); *rmin receives the smallest radius reached. */
/* Threads of the OpenMP loops, for timing the oracle on a chosen number of
 * host cores.  Every parallel loop writes disjoint outputs or reduces
 * integers, so results do not depend on the count. */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_kerr_fate(double a, double incl, double alpha, double beta, double* rmin) {
    const double si = sin(incl), ci = cos(incl);
    const double r_plus = 1.0 + sqrt(1.0 - a * a);
    const double s_cap = 1.0 / (r_plus + CAPTURE_CUSHION);
    kerr_par p;
    kerr_setup(&p, a, -alpha * si, (alpha * alpha - a * a) * ci * ci + beta * beta);
    double y[NSTATE] = {0.0, 1.0, ci, beta * si, 0.0, 0.0};
    double h = 1e-4, smax = 0.0;
    for (long steps = 0; steps < 20000000; ++steps) {
        double y5[NSTATE];
        const double err = dp_step(&p, y, h, y5, 1e-12, 1e-12);
        if (err > 1.0) { h *= fmax(0.2, 0.9 * pow(err, -0.2)); continue; }
        memcpy(y, y5, sizeof y);
        if (y[0] > smax) smax = y[0];
        if (y[0] >= s_cap) { *rmin = 1.0 / smax; return -1; }
        if (y[0] <= 0.0 || (y[1] < 0.0 && y[0] < 1e-3)) { *rmin = 1.0 / smax; return 1; }
        h *= fmin(5.0, fmax(0.2, 0.9 * pow(fmax(err, 1e-10), -0.2)));
        if (h > 0.02) h = 0.02;
    }
    *rmin = 1.0 / smax;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Schwarzschild: exact orbit integrals in u = 1/r with                      */
/*   (du/dpsi)^2 = P3(u) = 1/b^2 - u^2 + 2 u^3 ,                              */
/*   |dt/du| = 1 / (u^2 (1-2u) b sqrt(P3)).                                   */
/* The sweep angle psi from the observer direction is an incomplete elliptic */
/* integral of the first kind, evaluated with Carlson's R_F (Carlson 1995,   */
/* duplication algorithm, and the cubic reduction of DLMF 19.29.4).  The     */
/* time integral is evaluated by adaptive Gauss-Kronrod quadrature after a  */
/* substitution that removes the turning-point square-root singularity.      */
/* ------------------------------------------------------------------------ */
static double carlson_rf(double x, double y, double z) {
    for (int it = 0; it < 60; ++it) {
        const double A = (x + y + z) / 3.0;
        const double dev = fmax(fabs(A - x), fmax(fabs(A - y), fabs(A - z)));
        if (dev < 1e-4 * fabs(A)) break;
        const double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
        const double l = sx * sy + sy * sz + sz * sx;
        x = 0.25 * (x + l);
        y = 0.25 * (y + l);
        z = 0.25 * (z + l);
    }
    const double A = (x + y + z) / 3.0;
    const double X = 1.0 - x / A, Y = 1.0 - y / A, Z = -(X + Y);
    const double E2 = X * Y - Z * Z, E3 = X * Y * Z;
    return (1.0 - E2 / 10.0 + E3 / 14.0 + E2 * E2 / 24.0 - 3.0 * E2 * E3 / 44.0) / sqrt(A);
}

/* exported for the test that pins R_F against quadrature */
double orc_carlson_rf(double x, double y, double z) { return carlson_rf(x, y, z); }

/* Gauss-Kronrod 7-15 nodes/weights on [-1,1] (published constants). */
static const double GK_X[8] = {0.991455371120812639206854697526329,
                               0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926,
                               0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013,
                               0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245,
                               0.000000000000000000000000000000000};
static const double GK_WK[8] = {0.022935322010529224963732008058970,
                                0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518,
                                0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550,
                                0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649,
                                0.209482141084727828012999174891714};
static const double GK_WG[4] = {0.129484966168869693270611432679082,
                                0.279705391489276667901467771423780,
                                0.381830050505118944950369775488975,
                                0.417959183673469387755102040816327};

typedef double (*fn1)(double, const void*);

static double gk15(fn1 f, const void* ctx, double lo, double hi, double* err, double* absv) {
    const double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
    const double fc = f(c, ctx);
    double rk = fc * GK_WK[7], rg = fc * GK_WG[3], ra = fabs(fc) * GK_WK[7];
    for (int j = 0; j < 7; ++j) {
        const double dx = h * GK_X[j];
        const double f1 = f(c - dx, ctx), f2 = f(c + dx, ctx);
        rk += GK_WK[j] * (f1 + f2);
        ra += GK_WK[j] * (fabs(f1) + fabs(f2));
        if (j % 2 == 1) rg += GK_WG[j / 2] * (f1 + f2);
    }
    *err = fabs((rk - rg) * h);
    *absv = ra * fabs(h);
    return rk * h;
}

/* Adaptive bisection of GK15 panels.  tol is an absolute error target for
   the panel; a panel is also accepted once its error estimate reaches the
   rounding level of the integral of |f| over it, so the recursion stops. */
static double gk_adapt(fn1 f, const void* ctx, double lo, double hi, double tol, int depth) {
    double err, absv;
    const double v = gk15(f, ctx, lo, hi, &err, &absv);
    if (err <= tol || err <= 200.0 * 2.2e-16 * absv || depth >= 25) return v;
    const double m = 0.5 * (lo + hi);
    return gk_adapt(f, ctx, lo, m, 0.5 * tol, depth + 1) +
           gk_adapt(f, ctx, m, hi, 0.5 * tol, depth + 1);
}

/* relative-tolerance driver: the target is rel * |first estimate| */
static double gk_integrate(fn1 f, const void* ctx, double lo, double hi, double rel) {
    double err, absv;
    const double v0 = gk15(f, ctx, lo, hi, &err, &absv);
    return gk_adapt(f, ctx, lo, hi, rel * fabs(v0) + 1e-300, 0);
}

typedef struct {
    double b;
    double u1, u2, u3;   /* real roots u1 < 0 < u2 <= u3 (scattered rays) */
    double ut, us;       /* substitution end points */
    int scattered;
} schw_ray;

static double P3(double b, double u) { return 1.0 / (b * b) - u * u + 2.0 * u * u * u; }

/* integrand of psi for captured rays */
static double f_psi(double u, const void* c) {
    const schw_ray* s = (const schw_ray*)c;
    return 1.0 / sqrt(P3(s->b, u));
}

/* h(u) = |dt/du| - 1/u^2 - 2/u without cancellation (Q = b^2 P3):
   h = [b^2 (1-2u)/(1+sqrt Q) + 4 sqrt Q] / ((1-2u) sqrt Q) */
static double h_of(double b, double u, double sqQ) {
    return (b * b * (1.0 - 2.0 * u) / (1.0 + sqQ) + 4.0 * sqQ) / ((1.0 - 2.0 * u) * sqQ);
}

static double f_h_direct(double u, const void* c) {
    const schw_ray* s = (const schw_ray*)c;
    const double sqQ = s->b * sqrt(P3(s->b, u));
    return h_of(s->b, u, sqQ);
}

/* substituted integrands on w in [0,1]: u = ut - (ut-us) w^2, the factor w
   of du cancels the sqrt(ut - u) of P3 = 2 (u-u1)(u2-u)(u3-u). */
static double f_h_sub(double w, const void* c) {
    const schw_ray* s = (const schw_ray*)c;
    const double L = s->ut - s->us;
    const double u = s->ut - L * w * w;
    const double rest = sqrt(2.0 * (u - s->u1) * (s->u3 - u));  /* sqrt(P3)/(sqrt(L) w) */
    const double sqQ = s->b * rest * sqrt(L) * w;
    const double num = s->b * s->b * (1.0 - 2.0 * u) / (1.0 + sqQ) + 4.0 * sqQ;
    return 2.0 * sqrt(L) * num / ((1.0 - 2.0 * u) * s->b * rest);
}

static double f_g_sub(double w, const void* c) {
    const schw_ray* s = (const schw_ray*)c;
    const double L = s->ut - s->us;
    const double u = s->ut - L * w * w;
    const double rest = sqrt(2.0 * (u - s->u1) * (s->u3 - u));
    return 2.0 * sqrt(L) / (u * u * (1.0 - 2.0 * u) * s->b * rest);
}

/* psi(u) = int_0^u du / sqrt(P3) for a scattered ray, 0 <= u <= u2 */
static double psi_scat(const schw_ray* s, double x) {
    if (x <= 0.0) return 0.0;
    const double X1 = sqrt(x - s->u1), X2 = sqrt(fmax(s->u2 - x, 0.0)), X3 = sqrt(s->u3 - x);
    const double Y1 = sqrt(-s->u1), Y2 = sqrt(s->u2), Y3 = sqrt(s->u3);
    const double U12 = (X1 * X2 * Y3 + Y1 * Y2 * X3) / x;
    const double U13 = (X1 * X3 * Y2 + Y1 * Y3 * X2) / x;
    const double U23 = (X2 * X3 * Y1 + Y2 * Y3 * X1) / x;
    /* int dt / sqrt((t-u1)(u2-t)(u3-t)) = 2 R_F(U12^2, U13^2, U23^2); P3 has the factor 2 */
    return 2.0 * carlson_rf(U12 * U12, U13 * U13, U23 * U23) / sqrt(2.0);
}

static double polish_root(double b, double u) {
    for (int i = 0; i < 6; ++i) {
        const double f = P3(b, u), d = -2.0 * u + 6.0 * u * u;
        if (d == 0.0) break;
        u -= f / d;
    }
    return u;
}

static double psi_capt(const schw_ray* s, double u) {
    return gk_integrate(f_psi, s, 0.0, u, 1e-14);
}

/* Solve psi(u) = target for u in [0, umax] by bisection (psi monotone). */
static double invert_psi(const schw_ray* s, double target, double umax) {
    double lo = 0.0, hi = umax;
    for (int it = 0; it < 200; ++it) {
        const double m = 0.5 * (lo + hi);
        const double v = s->scattered ? psi_scat(s, m) : psi_capt(s, m);
        if (v < target) lo = m; else hi = m;
        if (hi - lo <= 1e-17) break;
    }
    return 0.5 * (lo + hi);
}

long orc_trace_schw(double incl, long n_rays, const double* alpha, const double* beta,
                    int n_orders, double r_esc, double* r_out, double* phi_out,
                    double* T_out, double* sr_out, int8_t* found) {
    (void)r_esc;
    const double si = sin(incl), ci = cos(incl), ti = tan(incl);
    const double u_cap = 1.0 / (2.0 + CAPTURE_CUSHION);
#pragma omp parallel for schedule(dynamic, 16)
    for (long ir = 0; ir < n_rays; ++ir) {
        const double al = alpha[ir], be = beta[ir];
        const double b = sqrt(al * al + be * be);
        for (int n = 0; n < n_orders; ++n) {
            const long o = ir * n_orders + n;
            found[o] = 0; r_out[o] = NAN; phi_out[o] = NAN; T_out[o] = NAN; sr_out[o] = 0.0;
        }
        if (b < 1e-12) continue;
        schw_ray s;
        memset(&s, 0, sizeof s);
        s.b = b;
        s.scattered = (b * b > 27.0);
        double psi_end, psi_t = 0.0;
        if (s.scattered) {
            const double th = acos(fmax(-1.0, fmin(1.0, 1.0 - 54.0 / (b * b))));
            s.u3 = polish_root(b, 1.0 / 6.0 + cos(th / 3.0) / 3.0);
            s.u2 = polish_root(b, 1.0 / 6.0 + cos(th / 3.0 - 2.0 * M_PI / 3.0) / 3.0);
            s.u1 = polish_root(b, 1.0 / 6.0 + cos(th / 3.0 + 2.0 * M_PI / 3.0) / 3.0);
            psi_t = psi_scat(&s, s.u2);
            psi_end = 2.0 * psi_t;
        } else {
            psi_end = psi_capt(&s, u_cap);
        }
        /* first equatorial crossing: cos i cos psi + (beta/b) sin i sin psi = 0 */
        const double psi0 = 0.5 * M_PI + atan((be / b) * ti);
        /* H(u_t) = int_0^{u_t} h du (scattered rays) */
        double H_t = 0.0;
        if (s.scattered) {
            s.ut = s.u2; s.us = 0.0;
            H_t = gk_integrate(f_h_sub, &s, 0.0, 1.0, 1e-14);
        }
        for (int n = 0; n < n_orders; ++n) {
            const double psin = psi0 + n * M_PI;
            if (psin >= psi_end) break;
            double u, T, sr;
            if (!s.scattered) {
                u = invert_psi(&s, psin, u_cap);
                const double H = gk_integrate(f_h_direct, &s, 0.0, u, 1e-14);
                T = H - (1.0 / u - 2.0 * log(u));
                sr = 1.0;
            } else if (psin <= psi_t) {
                u = invert_psi(&s, psin, s.u2);
                s.ut = s.u2; s.us = u;
                const double J = gk_integrate(f_h_sub, &s, 0.0, 1.0, 1e-14);
                T = (H_t - J) - (1.0 / u - 2.0 * log(u));
                sr = 1.0;
            } else {
                u = invert_psi(&s, 2.0 * psi_t - psin, s.u2);
                s.ut = s.u2; s.us = u;
                const double G = gk_integrate(f_g_sub, &s, 0.0, 1.0, 1e-14);
                T = H_t - (1.0 / s.u2 - 2.0 * log(s.u2)) + G;
                sr = -1.0;
            }
            if (!(u > 0.0)) break;
            const long o = ir * n_orders + n;
            found[o] = 1;
            r_out[o] = 1.0 / u;
            T_out[o] = T;
            sr_out[o] = sr;
            /* emission direction n = o cos psi + e sin psi projected on the plane */
            const double nx = si * cos(psin) - (be / b) * ci * sin(psin);
            const double ny = (al / b) * sin(psin);
            double ph = atan2(ny, nx);
            if (ph < 0.0) ph += 2.0 * M_PI;
            phi_out[o] = ph;
        }
    }
    return 0;
}

/* exported quadrature helpers for the pins */
typedef struct { double b; } psi_ctx;
static double f_psi_plain(double u, const void* c) {
    const psi_ctx* p = (const psi_ctx*)c;
    return 1.0 / sqrt(P3(p->b, u));
}
/* psi(u) for a scattered ray by the closed form (R_F) */
double orc_schw_psi(double b, double u) {
    schw_ray s;
    memset(&s, 0, sizeof s);
    s.b = b;
    const double th = acos(fmax(-1.0, fmin(1.0, 1.0 - 54.0 / (b * b))));
    s.u3 = polish_root(b, 1.0 / 6.0 + cos(th / 3.0) / 3.0);
    s.u2 = polish_root(b, 1.0 / 6.0 + cos(th / 3.0 - 2.0 * M_PI / 3.0) / 3.0);
    s.u1 = polish_root(b, 1.0 / 6.0 + cos(th / 3.0 + 2.0 * M_PI / 3.0) / 3.0);
    return psi_scat(&s, u);
}
/* same integral by brute-force adaptive quadrature (u below the turning point) */
double orc_schw_psi_quad(double b, double u) {
    psi_ctx c = {b};
    return gk_integrate(f_psi_plain, &c, 0.0, u, 1e-15);
}
double orc_schw_turning_u(double b) {
    const double th = acos(fmax(-1.0, fmin(1.0, 1.0 - 54.0 / (b * b))));
    return polish_root(b, 1.0 / 6.0 + cos(th / 3.0 - 2.0 * M_PI / 3.0) / 3.0);
}

/* ------------------------------------------------------------------------ */
/* Operator: y[row][f][b] = scale * sum_{e in row} w_e sum_c bil_c(e)        */
/*           sum_k B_k(t_o(f) - Delta_e) x[node_c(e)][k][b]                  */
/* (Eq. 2 per ray, Eq. 3 stacked by order, Eq. 16 whitened weight, Eq. 47). */
/* Source grid: N_r radii log-spaced on [r_in, r_out], N_phi azimuths        */
/* phi_j = 2 pi j / N_phi (periodic); bilinear in (log r, phi).              */
/* Hats: B_k(t) = max(0, 1 - |t - t_k| / dh), t_k = t_end - dh k.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n_r, n_phi;
    double r_in, r_out;
    int n_frames;
    double t0, cadence;
    int n_hats;
    double hat_step, t_end;
} orc_grid;

static void bilinear(const orc_grid* g, double r, double phi, long node[4], double wt[4]) {
    double rho = (log(r) - log(g->r_in)) / (log(g->r_out) - log(g->r_in)) * (g->n_r - 1);
    int i0 = (int)floor(rho);
    if (i0 < 0) i0 = 0;
    if (i0 > g->n_r - 2) i0 = g->n_r - 2;
    const double fr = rho - i0;
    double ph = phi / (2.0 * M_PI) * g->n_phi;
    ph = fmod(ph, (double)g->n_phi);
    if (ph < 0.0) ph += g->n_phi;
    int j0 = (int)floor(ph);
    if (j0 >= g->n_phi) j0 = g->n_phi - 1;
    const double fp = ph - j0;
    const int j1 = (j0 + 1) % g->n_phi;
    node[0] = (long)i0 * g->n_phi + j0;       wt[0] = (1.0 - fr) * (1.0 - fp);
    node[1] = (long)(i0 + 1) * g->n_phi + j0; wt[1] = fr * (1.0 - fp);
    node[2] = (long)i0 * g->n_phi + j1;       wt[2] = (1.0 - fr) * fp;
    node[3] = (long)(i0 + 1) * g->n_phi + j1; wt[3] = fr * fp;
}

/* BF16-weight tables (a precision option of the GPU tables, not of the
   paper): each corner weight W_c = (scale w) times its two bilinear factors,
   multiplied in the order (scale w) * a_c * b_c, is rounded to the nearest
   float and then to the nearest BF16 (8 significant bits, ties to even).   */
double orc_round_bf16(double v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

/* corner weights of one ray: wt[c] = scale w bil_c (FP64), or the BF16 weights */
static void corner_weights(const orc_grid* g, double r, double phi, double sw, int bf16,
                           long node[4], double wt[4]) {
    double bw[4];
    bilinear(g, r, phi, node, bw);
    if (!bf16) {
        for (int c = 0; c < 4; ++c) wt[c] = sw * bw[c];
        return;
    }
    /* the two factors of each corner, recovered from the stencil */
    double rho = (log(r) - log(g->r_in)) / (log(g->r_out) - log(g->r_in)) * (g->n_r - 1);
    int i0 = (int)floor(rho);
    if (i0 < 0) i0 = 0;
    if (i0 > g->n_r - 2) i0 = g->n_r - 2;
    const double fr = rho - i0;
    double ph = phi / (2.0 * M_PI) * g->n_phi;
    ph = fmod(ph, (double)g->n_phi);
    if (ph < 0.0) ph += g->n_phi;
    int j0 = (int)floor(ph);
    if (j0 >= g->n_phi) j0 = g->n_phi - 1;
    const double fp = ph - j0;
    wt[0] = orc_round_bf16(sw * (1.0 - fr) * (1.0 - fp));
    wt[1] = orc_round_bf16(sw * fr * (1.0 - fp));
    wt[2] = orc_round_bf16(sw * (1.0 - fr) * fp);
    wt[3] = orc_round_bf16(sw * fr * fp);
}

static double hat(const orc_grid* g, int k, double t) {
    const double tk = g->t_end - g->hat_step * k;
    const double v = 1.0 - fabs(t - tk) / g->hat_step;
    return v > 0.0 ? v : 0.0;
}

/* hats whose support can contain t (B_k(t) = 0 exactly for all others) */
static void hat_range(const orc_grid* g, double t, int* klo, int* khi) {
    const double u = (g->t_end - t) / g->hat_step;
    int lo = (int)floor(u) - 1, hi = (int)floor(u) + 2;
    if (lo < 0) lo = 0;
    if (hi > g->n_hats - 1) hi = g->n_hats - 1;
    *klo = lo; *khi = hi;
}

/* Rays are sorted by row; row_ptr[row]..row_ptr[row+1] are the rays (sub-rays
   of one pixel of one order) that form the pixel-average datum of that row. */
void orc_apply_A(const orc_grid* g, long n_rows, const int64_t* row_ptr, const double* r,
                     const double* phi, const double* delay, const double* w, double scale,
                     int bf16, int B, const double* x, double* y) {
    const int T = g->n_frames, K = g->n_hats;
    memset(y, 0, sizeof(double) * (size_t)n_rows * T * B);
#pragma omp parallel for schedule(dynamic, 32)
    for (long row = 0; row < n_rows; ++row) {
        for (long e = row_ptr[row]; e < row_ptr[row + 1]; ++e) {
            long node[4];
            double wt[4];
            corner_weights(g, r[e], phi[e], scale * w[e], bf16, node, wt);
            for (int f = 0; f < T; ++f) {
                const double t = g->t0 + g->cadence * f - delay[e];
                int klo, khi;
                hat_range(g, t, &klo, &khi);
                double* yy = y + ((size_t)row * T + f) * B;
                for (int c = 0; c < 4; ++c) {
                    for (int k = klo; k <= khi; ++k) {
                        const double hv = hat(g, k, t);
                        if (hv == 0.0) continue;
                        const double coef = wt[c] * hv;
                        const double* xx = x + ((size_t)node[c] * K + k) * B;
                        for (int b = 0; b < B; ++b) yy[b] += coef * xx[b];
                    }
                }
            }
        }
    }
}

/* exact transpose: x[node][k][b] = sum over (e, f, c) of the same coefficient
   times y[row(e)][f][b].  Parallel over (b, k) pairs, so every output element
   is accumulated by one thread in one fixed sequential order. */
void orc_apply_AT(const orc_grid* g, long n_rows, const int64_t* row_ptr, const double* r,
                  const double* phi, const double* delay, const double* w, double scale,
                  int bf16, int B, const double* y, double* x) {
    const int T = g->n_frames, K = g->n_hats;
    const long S = (long)g->n_r * g->n_phi;
    memset(x, 0, sizeof(double) * (size_t)S * K * B);
#pragma omp parallel for schedule(dynamic, 1)
    for (long task = 0; task < (long)B * K; ++task) {
        const int b = (int)(task / K), kk = (int)(task % K);
        for (long row = 0; row < n_rows; ++row) {
            for (long e = row_ptr[row]; e < row_ptr[row + 1]; ++e) {
                long node[4];
                double wt[4];
                corner_weights(g, r[e], phi[e], scale * w[e], bf16, node, wt);
                for (int f = 0; f < T; ++f) {
                    const double t = g->t0 + g->cadence * f - delay[e];
                    const double hv = hat(g, kk, t);
                    if (hv == 0.0) continue;
                    const double yv = y[((size_t)row * T + f) * B + b];
                    for (int c = 0; c < 4; ++c)
                        x[((size_t)node[c] * K + kk) * B + b] += wt[c] * hv * yv;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Scalar age probe (Eq. 10-12, Eq. 29):                                    */
/*   q_a(r, phi, t) = 1_[r_in, r_out](r) / N_h exp(-(t + a)^2 / (2 h^2))      */
/*   N_h^2 = pi (r_out^2 - r_in^2) h sqrt(pi)                                */
/*   I(a) = scale^2 sum_{rows, f} (sum_{e in row} w_e q_a(r_e, phi_e,        */
/*          t_o(f) - Delta_e))^2                                              */
/* evaluated directly at each ray's source point, not through the grid.     */
/* ------------------------------------------------------------------------ */
void orc_probe_info(const orc_grid* g, long n_rows, const int64_t* row_ptr, const double* r,
                    const double* delay, const double* w, double scale, double h, int n_ages,
                    const double* ages, double* info) {
    const int T = g->n_frames;
    const double Nh = sqrt(M_PI * (g->r_out * g->r_out - g->r_in * g->r_in) * h * sqrt(M_PI));
#pragma omp parallel for schedule(dynamic, 1)
    for (int ia = 0; ia < n_ages; ++ia) {
        const double a = ages[ia];
        double acc = 0.0;
        for (long row = 0; row < n_rows; ++row) {
            for (int f = 0; f < T; ++f) {
                double v = 0.0;
                for (long e = row_ptr[row]; e < row_ptr[row + 1]; ++e) {
                    const double t = g->t0 + g->cadence * f - delay[e];
                    const double ind = (r[e] >= g->r_in && r[e] <= g->r_out) ? 1.0 : 0.0;
                    v += w[e] * ind / Nh * exp(-(t + a) * (t + a) / (2.0 * h * h));
                }
                acc += v * v;
            }
        }
        info[ia] = scale * scale * acc;
    }
}
