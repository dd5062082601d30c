// Localized age probes (Sec. 3.3 Eq. 14): 28 directions
//   q_{a,l}(r, phi, t) = psi_l(r, phi) / N_{h,l} exp(-(t + a)^2 / (2 h^2)),
// psi_l = R_i(r) Phi_m(phi), l = 7 i + m: the cubic Bernstein polynomials in
// the log-radius coordinate times {1, cos phi, sin phi, ..., cos 3 phi,
// sin 3 phi}, each direction of unit L2 norm under r dr dphi dt.  The
// per-direction information I_l(a) = || scale A q_{a,l} ||^2 is the diagonal
// of the age-local Fisher matrix M(a) = P(a)^T P(a).
//
// Per row of the arm and age, with c_e = w_e psi_l(e) / N_{h,l} and g_e(f)
// the Gaussian at the ray's retarded time,
//   sum_f (sum_e c_e g_e(f))^2 = sum_{e, e'} c_e c_e' C_ee',
//   C_ee' = sum_f g_e(f) g_e'(f),
// so each (row, age) forms one small overlap matrix (one exponential per ray
// and frame; frames where every ray's exponent is below -100 are skipped, as
// in the scalar probe) and 28 quadratic forms.  FP64; a fixed grid per age
// and fixed-order reductions (bitwise repeatable).  Rows of more than four
// rays are not handled (RTT_ESTATE).
#include <cuda_runtime.h>

#include <cmath>

#include "rtt_internal.cuh"

namespace rtt {

constexpr int kLocDirs = 28;
constexpr int kLocMaxRays = 4;
constexpr int kLocBlocksX = 296;  // 2 x 148 blocks per age
constexpr int kLocThreads = 128;

struct LocNorm {
    double inv[kLocDirs];  // 1 / N_{h,l}
};

__device__ __forceinline__ int loc_arm_row(const ArmSeg& s, int row_out) {
    int r = row_out;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i < s.n && r < s.len[i]) return s.begin[i] + r;
        if (i < s.n) r -= s.len[i];
    }
    return -1;
}

// c[e][l] = w_e 1_[r_in, r_out](r_e) psi_l(r_e, phi_e) / N_{h,l}
__global__ void local_coef(int64_t E, const double* __restrict__ r, const double* __restrict__ phi,
                           const double* __restrict__ w, double r_in, double r_out, LocNorm nrm,
                           double* __restrict__ c) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const double re = r[e];
    const double ind = (re >= r_in && re <= r_out) ? 1.0 : 0.0;
    const double s = log(re / r_in) / log(r_out / r_in);
    const double u = 1.0 - s;
    const double R[4] = {u * u * u, 3.0 * s * u * u, 3.0 * s * s * u, s * s * s};
    const double p = phi[e];
    const double P[7] = {1.0, cos(p), sin(p), cos(2.0 * p), sin(2.0 * p), cos(3.0 * p), sin(3.0 * p)};
    const double we = w[e] * ind;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int m = 0; m < 7; ++m) c[e * kLocDirs + 7 * i + m] = we * R[i] * P[m] * nrm.inv[7 * i + m];
}

// block (x, age): rows ro = x * threads + t + k * (blocks * threads); partial
// sums of the 28 quadratic forms, reduced in a fixed order
__global__ void __launch_bounds__(kLocThreads)
local_probe(const int32_t* __restrict__ row_ptr, const double* __restrict__ delay,
            const double* __restrict__ coef, ArmSeg seg, int Tn, double t0, double cadence,
            double inv_2h2, double span, const double* __restrict__ ages, double* __restrict__ part,
            int* __restrict__ too_many) {
    const double a = ages[blockIdx.y];
    double sq[kLocDirs];
#pragma unroll
    for (int l = 0; l < kLocDirs; ++l) sq[l] = 0.0;
    for (int ro = blockIdx.x * blockDim.x + threadIdx.x; ro < seg.total; ro += gridDim.x * blockDim.x) {
        const int row = loc_arm_row(seg, ro);
        const int e0 = row_ptr[row], n = row_ptr[row + 1] - e0;
        if (n > kLocMaxRays) {
            atomicOr(too_many, 1);  // flag only: the result is rejected on the host
            continue;
        }
        double dl[kLocMaxRays];
        double dmin = 1e300, dmax = -1e300;
#pragma unroll
        for (int k = 0; k < kLocMaxRays; ++k) {
            dl[k] = k < n ? delay[e0 + k] : 0.0;
            if (k < n) {
                dmin = fmin(dmin, dl[k]);
                dmax = fmax(dmax, dl[k]);
            }
        }
        // frames with t_o(f) - Delta + a inside (-span, span) for some ray
        int f_lo = (int)floor((dmin - a - span - t0) / cadence) - 1;
        int f_hi = (int)ceil((dmax - a + span - t0) / cadence) + 1;
        f_lo = max(f_lo, 0);
        f_hi = min(f_hi, Tn - 1);
        double C[kLocMaxRays * (kLocMaxRays + 1) / 2];
#pragma unroll
        for (int k = 0; k < kLocMaxRays * (kLocMaxRays + 1) / 2; ++k) C[k] = 0.0;
        for (int f = f_lo; f <= f_hi; ++f) {
            const double t = t0 + cadence * f;
            double g[kLocMaxRays];
#pragma unroll
            for (int k = 0; k < kLocMaxRays; ++k) {
                const double d = t - dl[k] + a;
                const double arg = d * d * inv_2h2;
                g[k] = (k < n && arg < 100.0) ? exp(-arg) : 0.0;
            }
            int q = 0;
#pragma unroll
            for (int k = 0; k < kLocMaxRays; ++k)
#pragma unroll
                for (int k2 = k; k2 < kLocMaxRays; ++k2) C[q++] += g[k] * g[k2];
        }
        int q = 0;
#pragma unroll
        for (int k = 0; k < kLocMaxRays; ++k)
#pragma unroll
            for (int k2 = k; k2 < kLocMaxRays; ++k2) {
                if (k2 < n) {
                    const double m = (k == k2 ? 1.0 : 2.0) * C[q];
                    const double* ck = coef + (int64_t)(e0 + k) * kLocDirs;
                    const double* ck2 = coef + (int64_t)(e0 + k2) * kLocDirs;
#pragma unroll
                    for (int l = 0; l < kLocDirs; ++l) sq[l] += m * ck[l] * ck2[l];
                }
                ++q;
            }
    }
    // warp sums per direction, then the block's warps in order
    __shared__ double wsum[kLocThreads / 32][kLocDirs];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < kLocDirs; ++l) {
        double v = sq[l];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) wsum[warp][l] = v;
    }
    __syncthreads();
    if (threadIdx.x < kLocDirs) {
        double v = 0.0;
        for (int k = 0; k < kLocThreads / 32; ++k) v += wsum[k][threadIdx.x];
        part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * kLocDirs + threadIdx.x] = v;
    }
}

__global__ void local_reduce(int n_ages, int nbx, double scale2, const double* __restrict__ part,
                             double* __restrict__ info) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (age, direction)
    if (i >= n_ages * kLocDirs) return;
    const int a = i / kLocDirs, l = i - a * kLocDirs;
    double v = 0.0;
    for (int b = 0; b < nbx; ++b) v += part[((int64_t)a * nbx + b) * kLocDirs + l];
    info[i] = scale2 * v;
}

// N_{h,l}: int_{r_in}^{r_out} R_i(r)^2 r dr by composite Simpson in the
// log-radius coordinate (r = r_in e^{L s}, dr = L r ds), times int Phi_m^2
// dphi (2 pi for the constant, pi otherwise) and h sqrt(pi)
static LocNorm local_norms(double r_in, double r_out, double h) {
    const double L = std::log(r_out / r_in);
    const int n = 8192;
    double rad[4] = {0, 0, 0, 0};
    for (int k = 0; k <= n; ++k) {
        const double s = (double)k / n, u = 1.0 - s;
        const double wk = (k == 0 || k == n) ? 1.0 : (k % 2 ? 4.0 : 2.0);
        const double r = r_in * std::exp(L * s);
        const double R[4] = {u * u * u, 3.0 * s * u * u, 3.0 * s * s * u, s * s * s};
        for (int i = 0; i < 4; ++i) rad[i] += wk * R[i] * R[i] * r * r * L;
    }
    LocNorm nrm;
    for (int i = 0; i < 4; ++i) {
        rad[i] *= 1.0 / (3.0 * n);
        for (int m = 0; m < 7; ++m) {
            const double az = m == 0 ? 2.0 * M_PI : M_PI;
            nrm.inv[7 * i + m] = 1.0 / std::sqrt(rad[i] * az * h * std::sqrt(M_PI));
        }
    }
    return nrm;
}

}  // namespace rtt

using namespace rtt;

extern "C" rtt_status rtt_probe_info_local(rtt_op op, int arm_mask, int n_ages, const double* ages_host,
                                           double h, double* info_host, void* stream) {
    if (!op || !ages_host || !info_host || n_ages < 1 || n_ages > 4096 || !(h > 0.0)) {
        set_error("invalid localized-probe arguments (n_ages=%d h=%g)", n_ages, h);
        return RTT_EINVAL;
    }
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s != RTT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t E = op->n_rays;
    double *coef = nullptr, *ages = nullptr, *part = nullptr, *info = nullptr;
    int* flag = nullptr;
    cudaError_t e = cudaMalloc(&coef, (size_t)E * kLocDirs * 8);
    if (e == cudaSuccess) e = cudaMalloc(&ages, (size_t)n_ages * 8);
    if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)n_ages * kLocBlocksX * kLocDirs * 8);
    if (e == cudaSuccess) e = cudaMalloc(&info, (size_t)n_ages * kLocDirs * 8);
    if (e == cudaSuccess) e = cudaMalloc(&flag, 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ages, ages_host, (size_t)n_ages * 8, cudaMemcpyHostToDevice, st);
    int too_many = 0;
    if (e == cudaSuccess) {
        const LocNorm nrm = local_norms(op->grid.r_in, op->grid.r_out, h);
        local_coef<<<(int)((E + 255) / 256), 256, 0, st>>>(E, op->r, op->phi, op->weight, op->grid.r_in,
                                                           op->grid.r_out, nrm, coef);
        const double inv_2h2 = 1.0 / (2.0 * h * h);
        local_probe<<<dim3(kLocBlocksX, n_ages), kLocThreads, 0, st>>>(
            op->row_ptr, op->delay, coef, seg, op->time.n_frames, op->time.t0, op->time.cadence,
            inv_2h2, std::sqrt(100.0 / inv_2h2), ages, part, flag);
        local_reduce<<<(n_ages * kLocDirs + 255) / 256, 256, 0, st>>>(n_ages, kLocBlocksX,
                                                                      op->scale * op->scale, part, info);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(info_host, info, (size_t)n_ages * kLocDirs * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&too_many, flag, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    for (void* p : {(void*)coef, (void*)ages, (void*)part, (void*)info, (void*)flag})
        if (p) cudaFree(p);
    if (e != cudaSuccess) {
        set_error("localized probe information: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RTT_ENOMEM : RTT_ECUDA;
    }
    if (too_many) {
        set_error("localized probes: a row has more than %d rays", kLocMaxRays);
        return RTT_ESTATE;
    }
    return RTT_OK;
}
