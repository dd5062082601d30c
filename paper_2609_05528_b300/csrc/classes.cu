// Representation classes synthesised at the source nodes (Sec. 3.2 Eq. 5-8,
// Sec. 7): Q[(s, k)][c] = R_i(r_s) Phi_l(phi_s) tau_m(t_k),
// c = (i * 7 + l) * 8 + m, with
//   R_i: the 4 clamped cubic B-splines on uniform knots in log r (no interior
//        knots: cubic Bernstein polynomials of the normalised log radius),
//   Phi_l: 1, cos phi, sin phi, cos 2phi, sin 2phi, cos 3phi, sin 3phi,
//   tau_m: S224 - the 8 DCT-II modes cos(pi m (t - t_a) / (t_b - t_a)) on the
//          hat window [t_a, t_b] = [t_{K-1}, t_0]; L224 - 8 degree-one
//          B-splines on uniform knots over the same window.
#include <cuda_runtime.h>

#include <cmath>

#include "rtt_internal.cuh"

namespace rtt {

__global__ void synth_class_kernel(int n_r, int n_phi, int K, double t_end, double hat_step,
                                   int kind, double* Q) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n_r * n_phi * K * 224;
    if (t >= total) return;
    const int c = (int)(t % 224);
    const int64_t sk = t / 224;
    const int k = (int)(sk % K);
    const int64_t node = sk / K;
    const int ir = (int)(node / n_phi), jp = (int)(node - (int64_t)ir * n_phi);
    const int i = c / 56, l = (c / 8) % 7, m = c % 8;
    // radial: log-spaced nodes make the normalised log radius ir / (n_r - 1)
    const double s = (double)ir / (double)(n_r - 1);
    const double binom[4] = {1.0, 3.0, 3.0, 1.0};
    double R = binom[i];
    for (int q = 0; q < i; ++q) R *= s;
    for (int q = 0; q < 3 - i; ++q) R *= (1.0 - s);
    // azimuthal
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
    if (kind == 0) {
        tau = cos(3.141592653589793238462643383279 * m * (tk - ta) / (tb - ta));
    } else {
        const double step = (tb - ta) / 7.0;
        const double knot = ta + step * m;
        const double v = 1.0 - fabs(tk - knot) / step;
        tau = v > 0.0 ? v : 0.0;
    }
    Q[t] = R * Ph * tau;
}

}  // namespace rtt

using namespace rtt;

extern "C" rtt_status rtt_synth_class(rtt_op op, int kind, double* Q_dev, void* stream) {
    if (!op || !Q_dev || (kind != RTT_CLASS_S224 && kind != RTT_CLASS_L224)) {
        set_error("invalid class synthesis arguments (kind=%d)", kind);
        return RTT_EINVAL;
    }
    if (op->time.n_hats < 2) {
        set_error("class synthesis needs at least 2 hats (a non-empty time window)");
        return RTT_EINVAL;
    }
    const int64_t total = (int64_t)op->grid.n_r * op->grid.n_phi * op->time.n_hats * 224;
    synth_class_kernel<<<(int)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        op->grid.n_r, op->grid.n_phi, op->time.n_hats, op->time.t_end, op->time.hat_step, kind,
        Q_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("class synthesis: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    return RTT_OK;
}
