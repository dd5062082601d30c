// GPU null-geodesic tracer and raw ray-table assembly (Sec. 3.1 Eq. 2,
// Sec. 5: per-order source position, delay and transfer weight).
//
// One thread per screen sample integrates the Carter equations in Mino time
// with the regular variables s = 1/r and u = cos(theta):
//   (ds/dl)^2 = s^4 R(1/s),  (du/dl)^2 = eta - (eta + lam^2 - a^2) u^2 - a^2 u^4,
// written in second-order form (no sign flips at turning points), starting
// exactly at the observer (s = 0).  Classic RK4 with adaptive steps chosen by
// step doubling (Richardson error estimate, the extrapolated fifth-order
// state accepted); each sign change of u is refined by Newton iterations on
// the length of an extrapolated partial step.  The travel time is carried with the
// divergent r + 2 ln r part removed analytically.
#include <cuda_runtime.h>

#include <cmath>
#include <cub/cub.cuh>
#include <vector>

#include "rtt_internal.cuh"

namespace rtt {

struct RayConst {
    double a, lam, eta;
    double K;    // eta + (lam - a)^2
    double c2;   // 2 a^2 - 2 a lam - K
    double c0;   // (a^2 - a lam)^2 - a^2 K
    double m2;   // eta + lam^2 - a^2
};

struct St {
    double s, vs, u, vu, ph, Y;
};

__device__ __forceinline__ void deriv(const RayConst& c, const St& y, St& d) {
    const double s = y.s, s2 = s * s, u = y.u;
    const double a = c.a, a2 = a * a, al = a * c.lam;
    d.s = y.vs;
    d.vs = s * (c.c2 + s * (3.0 * c.K + 2.0 * c.c0 * s));
    d.u = y.vu;
    d.vu = -u * (c.m2 + 2.0 * a2 * u * u);
    const double del = 1.0 + s * (a2 * s - 2.0);              // Delta / r^2
    const double pe = 1.0 + (a2 - al) * s2;                    // (r^2 + a^2 - a lam) / r^2
    const double sn2 = 1.0 - u * u;
    d.ph = -(a * pe / del - a + c.lam / sn2);
    const double P = 1.0 + s2 * (c.c2 + s * (2.0 * c.K + c.c0 * s));
    const double rp = sqrt(fmax(P, 0.0));
    const double tail = al - a2 * sn2;
    if (y.vs >= 0.0) {
        // [ (1+a^2 s^2) pe - (1+2s) del sqrt(P) ] / s^2 without cancellation
        const double q = (c.c2 + s * (2.0 * c.K + c.c0 * s)) / (1.0 + rp);
        const double lead = (4.0 + a2 - al) + s * (-2.0 * a2 + (a2 * (a2 - al)) * s);
        d.Y = (lead - (1.0 + 2.0 * s) * del * q) / del + tail;
    } else {
        d.Y = ((1.0 + a2 * s2) * pe / del + (1.0 + 2.0 * s) * rp) / s2 + tail;
    }
}

__device__ __forceinline__ St axpy(const St& y, double h, const St& k) {
    return St{y.s + h * k.s, y.vs + h * k.vs, y.u + h * k.u, y.vu + h * k.vu, y.ph + h * k.ph,
              y.Y + h * k.Y};
}

// one step of h as two half steps, Richardson-extrapolated against the full
// step (fifth order); err receives the largest scaled local error estimate
__device__ __forceinline__ St rk4(const RayConst& c, const St& y, double h);

__device__ __forceinline__ St richardson_step(const RayConst& c, const St& y, double h, double tol,
                                              double* err) {
    const St full = rk4(c, y, h);
    const St half = rk4(c, rk4(c, y, 0.5 * h), 0.5 * h);
    const double e[6] = {half.s - full.s, half.vs - full.vs, half.u - full.u,
                         half.vu - full.vu, half.ph - full.ph, half.Y - full.Y};
    // error scales: every component relative to 1 + |value| except phi, which
    // is held absolutely (it grows by about 2 pi per order, its required
    // accuracy does not)
    const double m[6] = {1.0 + fmax(fabs(y.s), fabs(half.s)), 1.0 + fmax(fabs(y.vs), fabs(half.vs)),
                         1.0 + fmax(fabs(y.u), fabs(half.u)), 1.0 + fmax(fabs(y.vu), fabs(half.vu)),
                         1.0, 1.0 + fmax(fabs(y.Y), fabs(half.Y))};
    double er = 0.0;
    for (int q = 0; q < 6; ++q) er = fmax(er, fabs(e[q]) / (15.0 * tol * m[q]));
    *err = er;
    return St{half.s + e[0] / 15.0, half.vs + e[1] / 15.0, half.u + e[2] / 15.0,
              half.vu + e[3] / 15.0, half.ph + e[4] / 15.0, half.Y + e[5] / 15.0};
}

__device__ __forceinline__ St rk4(const RayConst& c, const St& y, double h) {
    St k1, k2, k3, k4;
    deriv(c, y, k1);
    deriv(c, axpy(y, 0.5 * h, k1), k2);
    deriv(c, axpy(y, 0.5 * h, k2), k3);
    deriv(c, axpy(y, h, k3), k4);
    const double h6 = h / 6.0;
    return St{y.s + h6 * (k1.s + 2.0 * (k2.s + k3.s) + k4.s),
              y.vs + h6 * (k1.vs + 2.0 * (k2.vs + k3.vs) + k4.vs),
              y.u + h6 * (k1.u + 2.0 * (k2.u + k3.u) + k4.u),
              y.vu + h6 * (k1.vu + 2.0 * (k2.vu + k3.vu) + k4.vu),
              y.ph + h6 * (k1.ph + 2.0 * (k2.ph + k3.ph) + k4.ph),
              y.Y + h6 * (k1.Y + 2.0 * (k2.Y + k3.Y) + k4.Y)};
}

struct TraceArgs {
    int64_t n;
    const double* alpha;
    const double* beta;
    const int32_t* n_sub;
    double a, sin_i, cos_i;
    double s_cap, s_esc;
    double r_in, r_out;
    double r_isco, E_isco, L_isco;
    double sqrt_domega, domega;
    double step_scale;
    double tol;
    // outputs, order-major [3][n]
    int32_t* valid;
    double* r;
    double* phi;
    double* T;
    double* w;
    double* thr;
    int32_t* status;  // per ray: 0 ok, 1 step limit
};

// Redshift factor g = 1 / (-p.u) of the emitter at radius r for a photon
// with (lam, eta) whose forward radial direction at emission is sr.
__device__ double redshift(const TraceArgs& A, double r, double lam, double eta, double sr) {
    const double a = A.a;
    if (r >= A.r_isco) {
        const double sq = sqrt(r);
        const double x = r * sq;  // r^{3/2}
        const double Om = 1.0 / (x + a);
        const double ut = (x + a) / (pow(r, 0.75) * sqrt(x - 3.0 * sq + 2.0 * a));
        return 1.0 / (ut * (1.0 - Om * lam));
    }
    const double E = A.E_isco, L = A.L_isco;
    const double r2 = r * r, del = r2 - 2.0 * r + a * a;
    const double P = E * (r2 + a * a) - a * L;
    const double ut = ((r2 + a * a) * P / del + a * (L - a * E)) / r2;
    const double up = (a * P / del + (L - a * E)) / r2;
    const double Rm = P * P - del * (r2 + (L - a * E) * (L - a * E));
    const double ur = -sqrt(fmax(Rm, 0.0)) / r2;
    const double Rph = (r2 + a * a - a * lam) * (r2 + a * a - a * lam) -
                       del * (eta + (lam - a) * (lam - a));
    const double pr = sr * sqrt(fmax(Rph, 0.0)) / del;
    return 1.0 / (ut - lam * up - pr * ur);
}

__global__ void trace_kernel(const TraceArgs A) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const double al = A.alpha[i], be = A.beta[i];
    RayConst c;
    c.a = A.a;
    c.lam = -al * A.sin_i;
    c.eta = (al * al - A.a * A.a) * A.cos_i * A.cos_i + be * be;
    c.K = c.eta + (c.lam - c.a) * (c.lam - c.a);
    c.c2 = 2.0 * c.a * c.a - 2.0 * c.a * c.lam - c.K;
    c.c0 = (c.a * c.a - c.a * c.lam) * (c.a * c.a - c.a * c.lam) - c.a * c.a * c.K;
    c.m2 = c.eta + c.lam * c.lam - c.a * c.a;
    const double rate = sqrt(fmax(fmax(fabs(c.c2), fabs(c.m2)), c.K));
    double h = A.step_scale / (1.0 + rate);
    St y{0.0, 1.0, A.cos_i, be * A.sin_i, 0.0, 0.0};
    int n_cross = 0;
    for (int n = 0; n < 3; ++n) A.valid[n * A.n + i] = 0;
    A.status[i] = 0;
    const double inv_nsub = 1.0 / (double)A.n_sub[i];
    // adaptive RK4 with step doubling: local error = (two half steps - one
    // full step) / 15 against tol (scaled as in richardson_step); the
    // accepted state is the Richardson-extrapolated one
    const double tol = A.tol;
    for (int step = 0; n_cross < 3; ++step) {
        if (step > 200000) {
            A.status[i] = 1;
            break;
        }
        double err = 0.0;
        const St yn = richardson_step(c, y, h, tol, &err);
        if (err > 1.0) {
            h *= fmax(0.1, 0.9 * pow(err, -0.2));
            continue;
        }
        if ((y.u > 0.0 && yn.u <= 0.0) || (y.u < 0.0 && yn.u >= 0.0)) {
            // the crossing u = 0 inside this step: Newton on the length of a
            // partial step from y, each partial step taken like an accepted
            // one (extrapolated, so of the same order)
            double hc = h * y.u / (y.u - yn.u), ec = 0.0;
            St yc = richardson_step(c, y, hc, tol, &ec);
            for (int it = 0; it < 8; ++it) {
                const double dh = -yc.u / yc.vu;
                hc += dh;
                yc = richardson_step(c, y, hc, tol, &ec);
                if (fabs(dh) < 1e-15 * h) break;
            }
            if (!(yc.s > 0.0 && yc.s < A.s_cap)) break;
            const double rr = 1.0 / yc.s;
            const int64_t o = n_cross * A.n + i;
            const bool ok = rr >= A.r_in && rr <= A.r_out;
            A.valid[o] = ok ? 1 : 0;
            double ph = fmod(yc.ph, 6.283185307179586476925286766559);
            if (ph < 0.0) ph += 6.283185307179586476925286766559;
            A.r[o] = rr;
            A.phi[o] = ph;
            A.T[o] = yc.Y - (rr + 2.0 * log(rr));
            const double sr = yc.vs >= 0.0 ? 1.0 : -1.0;
            const double g = redshift(A, rr, c.lam, c.eta, sr);
            const double g3 = g * g * g;
            A.w[o] = g3 * A.sqrt_domega * inv_nsub;
            A.thr[o] = g3 * A.domega * inv_nsub;
            ++n_cross;
        }
        y = yn;
        if (y.s >= A.s_cap) break;                  // captured
        if (y.vs < 0.0 && y.s < A.s_esc) break;     // outgoing beyond r_out
        if (y.s <= 0.0) break;                      // back at infinity
        h *= fmin(4.0, fmax(0.1, 0.9 * pow(fmax(err, 1e-12), -0.2)));
    }
}

__global__ void pack_keys(int64_t n3, int64_t n, const int32_t* valid, const int32_t* pixel,
                          unsigned long long* key, int32_t* idx, int32_t* flag) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n3) return;
    const int64_t order = t / n, i = t - order * n;
    key[t] = ((unsigned long long)order << 32) | (unsigned long long)(uint32_t)pixel[i];
    idx[t] = (int32_t)t;
    flag[t] = valid[t];
}

}  // namespace rtt

using namespace rtt;

static double isco_radius(double a) {
    const double z1 = 1.0 + std::cbrt(1.0 - a * a) * (std::cbrt(1.0 + a) + std::cbrt(1.0 - a));
    const double z2 = std::sqrt(3.0 * a * a + z1 * z1);
    return 3.0 + z2 - std::sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
}

extern "C" rtt_status rtt_trace_rays(const rtt_geometry* geom, const rtt_source_grid* grid,
                                     const rtt_screen* scr, rtt_ray_buffer* out, int64_t* n_out,
                                     void* stream) {
    if (!geom || !grid || !scr || !out || !n_out || !scr->alpha || !scr->beta || !scr->pixel ||
        !scr->n_sub) {
        set_error("null argument");
        return RTT_EINVAL;
    }
    const double a = geom->spin;
    if (!(std::fabs(a) < 1.0) || !(geom->incl_deg > 0.0 && geom->incl_deg < 90.0)) {
        set_error("geometry out of range (spin %g, incl %g)", a, geom->incl_deg);
        return RTT_EINVAL;
    }
    if (!(grid->r_in > 0.0) || !(grid->r_out > grid->r_in)) {
        set_error("invalid radial range");
        return RTT_EINVAL;
    }
    const int64_t n = scr->n;
    if (n < 1 || n > (1ll << 28) || out->capacity < 3 * n || !(scr->d_omega_pixel > 0.0)) {
        set_error("invalid screen size %lld or capacity %lld", (long long)n,
                  (long long)out->capacity);
        return RTT_EINVAL;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (scr->n_sub[i] < 1 || scr->pixel[i] < 0 || !std::isfinite(scr->alpha[i]) ||
            !std::isfinite(scr->beta[i])) {
            set_error("screen sample %lld invalid", (long long)i);
            return RTT_EINVAL;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<void*> bufs;
    auto cleanup = [&]() {
        for (void* p : bufs) cudaFree(p);
    };
    auto get = [&](void** p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes + 16) != cudaSuccess) return false;
        bufs.push_back(*p);
        return true;
    };
    double *d_al, *d_be, *d_r, *d_phi, *d_T, *d_w, *d_thr;
    int32_t *d_nsub, *d_pix, *d_valid, *d_status, *d_idx, *d_perm, *d_flag, *d_pos;
    unsigned long long *d_key, *d_key2;
    const int64_t n3 = 3 * n;
    bool ok = get((void**)&d_al, n * 8) && get((void**)&d_be, n * 8) &&
              get((void**)&d_nsub, n * 4) && get((void**)&d_pix, n * 4) &&
              get((void**)&d_r, n3 * 8) && get((void**)&d_phi, n3 * 8) &&
              get((void**)&d_T, n3 * 8) && get((void**)&d_w, n3 * 8) &&
              get((void**)&d_thr, n3 * 8) && get((void**)&d_valid, n3 * 4) &&
              get((void**)&d_status, n * 4) && get((void**)&d_idx, n3 * 4) &&
              get((void**)&d_perm, n3 * 4) && get((void**)&d_flag, n3 * 4) &&
              get((void**)&d_pos, n3 * 4) && get((void**)&d_key, n3 * 8) &&
              get((void**)&d_key2, n3 * 8);
    if (!ok) {
        cleanup();
        set_error("device allocation failed in rtt_trace_rays");
        return RTT_ENOMEM;
    }
#define TRY_CUDA(x)                                                               \
    do {                                                                          \
        cudaError_t _e = (x);                                                     \
        if (_e != cudaSuccess) {                                                  \
            set_error("%s failed: %s", #x, cudaGetErrorString(_e));               \
            cleanup();                                                            \
            return RTT_ECUDA;                                                     \
        }                                                                         \
    } while (0)
    TRY_CUDA(cudaMemcpyAsync(d_al, scr->alpha, n * 8, cudaMemcpyHostToDevice, st));
    TRY_CUDA(cudaMemcpyAsync(d_be, scr->beta, n * 8, cudaMemcpyHostToDevice, st));
    TRY_CUDA(cudaMemcpyAsync(d_nsub, scr->n_sub, n * 4, cudaMemcpyHostToDevice, st));
    TRY_CUDA(cudaMemcpyAsync(d_pix, scr->pixel, n * 4, cudaMemcpyHostToDevice, st));
    TraceArgs A{};
    A.n = n;
    A.alpha = d_al;
    A.beta = d_be;
    A.n_sub = d_nsub;
    A.a = a;
    const double inc = geom->incl_deg * M_PI / 180.0;
    A.sin_i = std::sin(inc);
    A.cos_i = std::cos(inc);
    const double r_plus = 1.0 + std::sqrt(1.0 - a * a);
    A.s_cap = 1.0 / (r_plus + 0.01);
    A.s_esc = 1.0 / grid->r_out;
    A.r_in = grid->r_in;
    A.r_out = grid->r_out;
    A.r_isco = isco_radius(a);
    {
        const double r = A.r_isco, sq = std::sqrt(r), x = r * sq;
        const double den = std::pow(r, 0.75) * std::sqrt(x - 3.0 * sq + 2.0 * a);
        A.E_isco = (x - 2.0 * sq + a) / den;
        A.L_isco = (r * r - 2.0 * a * sq + a * a) / den;
    }
    A.domega = scr->d_omega_pixel;
    A.sqrt_domega = std::sqrt(scr->d_omega_pixel);
    A.step_scale = 0.01;
    A.tol = 1e-14;
    A.valid = d_valid;
    A.r = d_r;
    A.phi = d_phi;
    A.T = d_T;
    A.w = d_w;
    A.thr = d_thr;
    A.status = d_status;
    trace_kernel<<<(int)((n + 127) / 128), 128, 0, st>>>(A);
    TRY_CUDA(cudaGetLastError());
    // compaction in (order, pixel, sample) order: stable sort of all
    // (order, sample) slots by key, then an exclusive scan of validity
    pack_keys<<<(int)((n3 + 255) / 256), 256, 0, st>>>(n3, n, d_valid, d_pix, d_key, d_idx,
                                                        d_flag);
    TRY_CUDA(cudaGetLastError());
    size_t tb = 0;
    TRY_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, d_key, d_key2, d_idx, d_perm, n3, 0, 34,
                                             st));
    void* d_tmp;
    if (!get(&d_tmp, tb)) {
        cleanup();
        set_error("device allocation failed in rtt_trace_rays");
        return RTT_ENOMEM;
    }
    TRY_CUDA(cub::DeviceRadixSort::SortPairs(d_tmp, tb, d_key, d_key2, d_idx, d_perm, n3, 0, 34,
                                             st));
    // host side gather of the sorted valid entries (the table is a host output)
    std::vector<int32_t> perm(n3), valid(n3), status(n);
    std::vector<double> r(n3), phi(n3), T(n3), w(n3), thr(n3);
    TRY_CUDA(cudaMemcpyAsync(perm.data(), d_perm, n3 * 4, cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(valid.data(), d_valid, n3 * 4, cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(status.data(), d_status, n * 4, cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(r.data(), d_r, n3 * 8, cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(phi.data(), d_phi, n3 * 8, cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(T.data(), d_T, n3 * 8, cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(w.data(), d_w, n3 * 8, cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaMemcpyAsync(thr.data(), d_thr, n3 * 8, cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaStreamSynchronize(st));
    cleanup();
#undef TRY_CUDA
    int64_t bad = 0;
    for (int64_t i = 0; i < n; ++i) bad += status[i] != 0;
    if (bad) {
        set_error("%lld rays hit the integrator step limit", (long long)bad);
        return RTT_ENOTCONVERGED;
    }
    double Tmin = INFINITY;
    for (int64_t i = 0; i < n; ++i)
        if (valid[i]) Tmin = std::fmin(Tmin, T[i]);
    if (!std::isfinite(Tmin)) {
        set_error("no valid direct ray");
        return RTT_EINVAL;
    }
    int64_t m = 0;
    for (int64_t t = 0; t < n3; ++t) {
        const int32_t s = perm[t];
        if (!valid[s]) continue;
        out->order[m] = (int8_t)(s / n);
        out->pixel[m] = scr->pixel[s % n];
        out->r[m] = r[s];
        out->phi[m] = phi[s];
        out->delay[m] = T[s] - Tmin;
        out->weight[m] = w[s];
        out->throughput[m] = thr[s];
        ++m;
    }
    *n_out = m;
    return RTT_OK;
}
