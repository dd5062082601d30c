// Representation classes synthesised at the source nodes (Sec. 3.2 Eq. 5-8,
// Sec. 7-8 Eq. 43): Q[(s, k)][c] = R_i(r_s) Phi_l(phi_s) tau_m(t_k),
// c = (i * NA + l) * NT + m, with
//   R_i: NR clamped cubic B-splines on uniform knots in log r (NR = 4: no
//        interior knot, the cubic Bernstein polynomials),
//   Phi_l: 1, cos phi, sin phi, cos 2phi, sin 2phi, ... (NA of them),
//   tau_m: S classes - the NT DCT-II modes cos(pi m (t - t_a) / (t_b - t_a))
//          on the hat window [t_a, t_b] = [t_{K-1}, t_0]; L classes - NT
//          degree-one B-splines on uniform knots over the same window.
// (NR, NA, NT): S224 / L224 (4, 7, 8); S448T / L448 (4, 7, 16); S528S
// (6, 11, 8); S1056ST / L1056 (6, 11, 16).
#include <cuda_runtime.h>

#include <cmath>

#include "rtt_internal.cuh"

namespace rtt {

// the ladder of Sec. 7-8 (Eq. 43): radial x real-azimuthal x temporal
// dimensions, temporal family (0 DCT-II modes, 1 degree-one B-splines)
struct ClassShape {
    int nr, na, nt, fam;
};
static bool class_shape(int kind, ClassShape* cs) {
    switch (kind) {
        case RTT_CLASS_S224: *cs = {4, 7, 8, 0}; return true;
        case RTT_CLASS_L224: *cs = {4, 7, 8, 1}; return true;
        case RTT_CLASS_S448T: *cs = {4, 7, 16, 0}; return true;
        case RTT_CLASS_S528S: *cs = {6, 11, 8, 0}; return true;
        case RTT_CLASS_S1056ST: *cs = {6, 11, 16, 0}; return true;
        case RTT_CLASS_L448: *cs = {4, 7, 16, 1}; return true;
        case RTT_CLASS_L1056: *cs = {6, 11, 16, 1}; return true;
        default: return false;
    }
}

// clamped cubic B-spline i of n on uniform knots over [0, 1] at s (Cox-de Boor)
__device__ double radial_bspline(int i, int n, double s) {
    double t[16];  // knots: 4 zeros, n - 4 uniform interior knots, 4 ones
    const int nk = n + 4;
    for (int k = 0; k < nk; ++k) {
        if (k < 4) t[k] = 0.0;
        else if (k >= n) t[k] = 1.0;
        else t[k] = (double)(k - 3) / (double)(n - 3);
    }
    // degree 0 on [t_j, t_{j+1}); the last non-empty interval is closed at 1
    double N[16];
    for (int j = 0; j < nk - 1; ++j) {
        const bool last = t[j] < t[j + 1] && t[j + 1] == 1.0;
        N[j] = ((s >= t[j] && s < t[j + 1]) || (last && s == 1.0)) ? 1.0 : 0.0;
    }
    for (int p = 1; p <= 3; ++p)
        for (int j = 0; j < nk - 1 - p; ++j) {
            const double d1 = t[j + p] - t[j], d2 = t[j + p + 1] - t[j + 1];
            const double a = d1 > 0.0 ? (s - t[j]) / d1 * N[j] : 0.0;
            const double b = d2 > 0.0 ? (t[j + p + 1] - s) / d2 * N[j + 1] : 0.0;
            N[j] = a + b;
        }
    return N[i];
}

__global__ void synth_class_kernel(int n_r, int n_phi, int K, double t_end, double hat_step,
                                   ClassShape cs, double* Q) {
    const int d = cs.nr * cs.na * cs.nt;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n_r * n_phi * K * d;
    if (t >= total) return;
    const int c = (int)(t % d);
    const int64_t sk = t / d;
    const int k = (int)(sk % K);
    const int64_t node = sk / K;
    const int ir = (int)(node / n_phi), jp = (int)(node - (int64_t)ir * n_phi);
    const int m = c % cs.nt, l = (c / cs.nt) % cs.na, i = c / (cs.nt * cs.na);
    // radial: log-spaced nodes make the normalised log radius ir / (n_r - 1)
    const double s = (double)ir / (double)(n_r - 1);
    double R;
    if (cs.nr == 4) {  // no interior knot: the cubic Bernstein polynomials
        const double binom[4] = {1.0, 3.0, 3.0, 1.0};
        R = binom[i];
        for (int q = 0; q < i; ++q) R *= s;
        for (int q = 0; q < 3 - i; ++q) R *= (1.0 - s);
    } else {
        R = radial_bspline(i, cs.nr, s);
    }
    // azimuthal: 1, cos phi, sin phi, cos 2 phi, ...
    const double phi = 6.283185307179586476925286766559 * (double)jp / (double)n_phi;
    double Ph = 1.0;
    if (l > 0) {
        const int mm = (l + 1) / 2;
        Ph = (l & 1) ? cos(mm * phi) : sin(mm * phi);
    }
    // temporal on [t_a, t_b] = [t_{K-1}, t_0]
    const double tk = t_end - hat_step * k;
    const double ta = t_end - hat_step * (K - 1), tb = t_end;
    double tau;
    if (cs.fam == 0) {
        tau = cos(3.141592653589793238462643383279 * m * (tk - ta) / (tb - ta));
    } else {
        const double step = (tb - ta) / (double)(cs.nt - 1);
        const double knot = ta + step * m;
        const double v = 1.0 - fabs(tk - knot) / step;
        tau = v > 0.0 ? v : 0.0;
    }
    Q[t] = R * Ph * tau;
}

}  // namespace rtt

using namespace rtt;

extern "C" int rtt_class_dim(int kind) {
    ClassShape cs;
    return class_shape(kind, &cs) ? cs.nr * cs.na * cs.nt : 0;
}

extern "C" rtt_status rtt_synth_class(rtt_op op, int kind, double* Q_dev, void* stream) {
    ClassShape cs;
    if (!op || !Q_dev || !class_shape(kind, &cs)) {
        set_error("invalid class synthesis arguments (kind=%d)", kind);
        return RTT_EINVAL;
    }
    if (op->time.n_hats < 2) {
        set_error("class synthesis needs at least 2 hats (a non-empty time window)");
        return RTT_EINVAL;
    }
    const int d = cs.nr * cs.na * cs.nt;
    const int64_t total = (int64_t)op->grid.n_r * op->grid.n_phi * op->time.n_hats * d;
    synth_class_kernel<<<(int)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        op->grid.n_r, op->grid.n_phi, op->time.n_hats, op->time.t_end, op->time.hat_step, cs, Q_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("class synthesis: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    return RTT_OK;
}
