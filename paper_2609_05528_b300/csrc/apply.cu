// Forward operator A and its adjoint A^T (Sec. 3.1 Eq. 2-3, Eq. 16, Eq. 47).
//
// Forward (one warp per (row, frame chunk, batch chunk)):
//   for each ray e of the row, the spatially interpolated history
//   z_e[k][b] = sum_c W_{e,c} x[node_c][k][b] is staged in shared memory for
//   the hats the frame chunk can touch, then every output sample adds
//   (1 - fr) z_e[k0] + fr z_e[k0 + 1] with the exact integer hat index k0 and
//   24-bit fraction fr of that (ray, frame).  y is written once, coalesced.
// Adjoint (one warp per (node, hat chunk, batch chunk)): a deterministic
//   gather over the node's incidence list (sorted by ray), summing for each
//   owned (k, b) the frames whose hat pair contains k, with the same integer
//   hat arithmetic as the forward, so the two are exact transposes.
#include <cuda_runtime.h>

#include "rtt_internal.cuh"

namespace rtt {

template <typename T>
struct HatCoef;

// FP32 path: fraction held as a 24-bit integer.
template <>
struct HatCoef<float> {
    int32_t K0, F0;
    int64_t D;
    __device__ __forceinline__ void at(int f, int& k0, float& fr) const {
        const int64_t fd = (int64_t)f * D;
        const int32_t A = (int32_t)(fd >> kFracBits);
        const int32_t R = (int32_t)(fd & kFracMask);
        int32_t F = F0 - R;
        k0 = K0 - A;
        if (F < 0) {
            F += kFracOne;
            k0 -= 1;
        }
        fr = (float)F * (1.0f / (float)kFracOne);
    }
};

// FP64 path: exact FP64 fraction; the per-frame offset f * delta is dyadic.
template <>
struct HatCoef<double> {
    int32_t K0;
    double F;
    int64_t D;
    __device__ __forceinline__ void at(int f, int& k0, double& fr) const {
        const int64_t fd = (int64_t)f * D;
        const int32_t A = (int32_t)(fd >> kFracBits);
        const double R = (double)(fd & kFracMask) * (1.0 / (double)kFracOne);
        double v = F - R;
        k0 = K0 - A;
        if (v < 0.0) {
            v += 1.0;
            k0 -= 1;
        }
        fr = v;
    }
};

template <typename T>
struct ApplyArgs {
    const int32_t* row_ptr;
    const int32_t* ray_row;
    const int32_t* row_order;
    const int32_t* node00;
    const int32_t* node01;
    const float4* W;
    const double* W64;
    const int32_t* K0;
    const int32_t* F0;
    const double* F64;
    const int32_t* node_ptr;
    const int32_t* inc;
    const T* in;
    T* out;
    int B, K, Tn, n_phi, n_nodes;
    int64_t D;
    double delta;
    ArmSeg seg;
    int FC;       // frames per chunk (forward)
    int zwin;     // hats staged per chunk (forward)
    int KC;       // hats per chunk (adjoint)
    int vec4;     // batch stride and chunk allow 16-byte loads
    T* zhat;      // adjoint scratch [E][K][Bc]
    int Bc;       // batch entries held per ray in zhat
    int64_t n_rays_total;
    int seg_rows_all;  // total rows of the operator (all orders)
    const int32_t* node_order;  // nodes by descending incidence count (load balance)
    int n_fchunk, n_bchunk, n_kchunk;
    int64_t n_tasks;
};

template <typename T>
__device__ __forceinline__ void load_w(const ApplyArgs<T>& a, int e, T w[4]);

template <>
__device__ __forceinline__ void load_w<float>(const ApplyArgs<float>& a, int e, float w[4]) {
    const float4 v = a.W[e];
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}
template <>
__device__ __forceinline__ void load_w<double>(const ApplyArgs<double>& a, int e, double w[4]) {
    const double2* p = reinterpret_cast<const double2*>(a.W64 + 4 * (int64_t)e);
    const double2 v0 = p[0], v1 = p[1];
    w[0] = v0.x; w[1] = v0.y; w[2] = v1.x; w[3] = v1.y;
}

template <typename T>
__device__ __forceinline__ HatCoef<T> load_hat(const ApplyArgs<T>& a, int e);
template <>
__device__ __forceinline__ HatCoef<float> load_hat<float>(const ApplyArgs<float>& a, int e) {
    HatCoef<float> h;
    h.K0 = a.K0[e]; h.F0 = a.F0[e]; h.D = a.D;
    return h;
}
template <>
__device__ __forceinline__ HatCoef<double> load_hat<double>(const ApplyArgs<double>& a, int e) {
    HatCoef<double> h;
    h.K0 = a.K0[e]; h.F = a.F64[e]; h.D = a.D;
    return h;
}

__device__ __forceinline__ int seg_in_row(const ArmSeg& s, int row_out) {
    int r = row_out;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i < s.n && r < s.len[i]) return s.begin[i] + r;
        if (i < s.n) r -= s.len[i];
    }
    return -1;
}

// output row of an input row under the arm mask, -1 if not selected
__device__ __forceinline__ int seg_out_row(const ArmSeg& s, int row_in) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i < s.n && row_in >= s.begin[i] && row_in < s.begin[i] + s.len[i])
            return s.out_off[i] + (row_in - s.begin[i]);
    }
    return -1;
}

constexpr int kWarpsPerBlock = 8;

constexpr int kAdjOutPerLane = 8;

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t d) {
    return a >= 0 ? a / d : -((-a + d - 1) / d);
}

// Phase 1 of the adjoint: temporal contraction per ray,
//   zhat_e[k][b] = sum_f h_{e,f,k} y[row_e][f][b0 + b],
// one warp per (ray, hat chunk, batch chunk).  The frames feeding hat k are
// the contiguous range where the exact hat index is k or k - 1, found by
// integer division on the 24-bit fixed-point hat coordinate.
template <typename T, int BC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
adj_time_kernel(const ApplyArgs<T> a) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t task = warp_global; task < a.n_tasks; task += n_warps) {
        const int bchunk = (int)(task % a.n_bchunk);
        const int64_t t2 = task / a.n_bchunk;
        const int kchunk = (int)(t2 % a.n_kchunk);
        const int e = (int)(t2 / a.n_kchunk);
        const int row_out = seg_out_row(a.seg, a.ray_row[e]);
        if (row_out < 0) {
            // rays outside the arm contribute nothing: their zhat rows are zero
            const int k_begin = kchunk * a.KC;
            for (int o = lane; o < a.KC * a.Bc; o += 32) {
                const int kk = o / a.Bc, bb = o - kk * a.Bc;
                if (k_begin + kk < a.K) a.zhat[((int64_t)e * a.K + k_begin + kk) * a.Bc + bb] = T(0);
            }
            continue;
        }
        const HatCoef<T> hc = load_hat(a, e);
        const int64_t U0 = (int64_t)a.K0[e] * kFracOne + (int64_t)a.F0[e];
        const T* yrow = a.in + (int64_t)row_out * a.Tn * a.B;
        const int b0 = bchunk * BC;
        const int k_begin = kchunk * a.KC;
#pragma unroll
        for (int j = 0; j < kAdjOutPerLane; ++j) {
            const int o = lane + 32 * j;
            const int kk = o / BC, bb = o - kk * BC;
            const int k = k_begin + kk;
            const int b = b0 + bb;
            if (kk >= a.KC || k >= a.K || bb >= a.Bc) continue;
            T s = T(0);
            if constexpr (sizeof(T) == 4) {
                // frames with (k-1) 2^24 <= U(f) < (k+1) 2^24, U(f) = U0 - f D:
                // start from a float estimate and test each frame exactly
                const int64_t hi_excl = (int64_t)(k + 1) * kFracOne;
                const int64_t lo_incl = (int64_t)(k - 1) * kFracOne;
                const float est = (float)(U0 - hi_excl) * (1.0f / (float)a.D);
                int f = (int)fminf(fmaxf(floorf(est) - 1.0f, 0.0f), (float)a.Tn);
                int64_t U = U0 - (int64_t)f * a.D;
                while (f < a.Tn && U >= hi_excl) { ++f; U -= a.D; }
                for (; f < a.Tn && U >= lo_incl; ++f, U -= a.D) {
                    const int k0 = (int)(U >> kFracBits);
                    const float fr = (float)(int32_t)(U & kFracMask) * (1.0f / (float)kFracOne);
                    const float hw = (k0 == k) ? 1.0f - fr : fr;
                    s += hw * yrow[(int64_t)f * a.B + b];
                }
            } else {
                int64_t flo = floor_div(U0 - (int64_t)(k + 1) * kFracOne, a.D) + 1;
                int64_t fhi = floor_div(U0 - (int64_t)(k - 1) * kFracOne, a.D);
                if (flo < 0) flo = 0;
                if (fhi > a.Tn - 1) fhi = a.Tn - 1;
                for (int f = (int)flo; f <= (int)fhi; ++f) {
                    int k0;
                    T fr;
                    hc.at(f, k0, fr);
                    const T hw = (k0 == k) ? T(1) - fr : ((k0 + 1 == k) ? fr : T(0));
                    s += hw * yrow[(int64_t)f * a.B + b];
                }
            }
            a.zhat[((int64_t)e * a.K + k) * a.Bc + bb] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Fast paths (FP32 and FP64 storage).  Forward: lane per frame, each lane
// carries all BC batch entries of its frames, so the exact hat index and
// fraction of a (ray, frame) are computed once and the staged z rows are read
// as 16-byte vectors.  FP32 takes the fraction from the 24-bit fixed-point
// hat coordinate; FP64 takes the exact FP64 fraction (same integer index).
// ---------------------------------------------------------------------------
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int W = 2; };

template <typename T>
__device__ __forceinline__ T* comps(typename Vec16<T>::type& v) { return reinterpret_cast<T*>(&v); }
template <typename T>
__device__ __forceinline__ const T* comps(const typename Vec16<T>::type& v) {
    return reinterpret_cast<const T*>(&v);
}

// hat fraction of a frame with fixed-point coordinate U = U0 - f D
template <typename T>
__device__ __forceinline__ T frac_of(int64_t U, int f, int64_t D, double F64);
template <>
__device__ __forceinline__ float frac_of<float>(int64_t U, int, int64_t, double) {
    return (float)(int32_t)(U & kFracMask) * (1.0f / (float)kFracOne);
}
template <>
__device__ __forceinline__ double frac_of<double>(int64_t, int f, int64_t D, double F64) {
    const double R = (double)(((int64_t)f * D) & kFracMask) * (1.0 / (double)kFracOne);
    const double v = F64 - R;
    return v < 0.0 ? v + 1.0 : v;
}

template <typename T>
__device__ __forceinline__ double exact_frac(const ApplyArgs<T>& a, int e);
template <>
__device__ __forceinline__ double exact_frac<float>(const ApplyArgs<float>&, int) { return 0.0; }
template <>
__device__ __forceinline__ double exact_frac<double>(const ApplyArgs<double>& a, int e) {
    return a.F64[e];
}

template <typename T>
__device__ __forceinline__ void corner_w(const ApplyArgs<T>& a, int e, T w[4]) { load_w(a, e, w); }

template <typename T, int BC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, (sizeof(T) == 8 || BC >= 32) ? 1 : 2)
fwd3_kernel(const ApplyArgs<T> a) {
    using V = typename Vec16<T>::type;
    constexpr int VW = Vec16<T>::W;
    constexpr int FPL = BC >= 32 ? 1 : 32 / BC;  // frames per lane
    constexpr int FC = 32 * FPL;                 // frames per task
    extern __shared__ __align__(16) unsigned char smem3_raw[];
    T* zs = reinterpret_cast<T*>(smem3_raw) + (threadIdx.x >> 5) * (a.zwin * BC);
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * kWarpsPerBlock;
    const bool vec = (BC >= VW) && a.vec4;
    for (int64_t task = warp_global; task < a.n_tasks; task += n_warps) {
        const int bchunk = (int)(task % a.n_bchunk);
        const int64_t t2 = task / a.n_bchunk;
        const int fchunk = (int)(t2 % a.n_fchunk);
        const int row_out = (int)(t2 / a.n_fchunk);
        const int row = seg_in_row(a.seg, row_out);
        const int f_begin = fchunk * FC;
        const int f_end = min(a.Tn, f_begin + FC);
        const int b0 = bchunk * BC;
        const int nb = min(BC, a.B - b0);
        T acc[FPL][BC];
#pragma unroll
        for (int j = 0; j < FPL; ++j)
#pragma unroll
            for (int b = 0; b < BC; ++b) acc[j][b] = T(0);
        const int e_begin = a.row_ptr[row], e_end = a.row_ptr[row + 1];
        for (int e = e_begin; e < e_end; ++e) {
            const int64_t U0 = (int64_t)a.K0[e] * kFracOne + (int64_t)a.F0[e];
            const double F64 = exact_frac(a, e);
            const int k_top = (int)((U0 - (int64_t)f_begin * a.D) >> kFracBits);
            const int k_lo = (int)((U0 - (int64_t)(f_end - 1) * a.D) >> kFracBits);
            const int nwin = k_top + 2 - k_lo;
            T w[4];
            corner_w(a, e, w);
            const int n00 = a.node00[e], n01 = a.node01[e];
            const int64_t KB = (int64_t)a.K * a.B;
            const T* x00 = a.in + (int64_t)n00 * KB + b0;
            const T* x10 = a.in + (int64_t)(n00 + a.n_phi) * KB + b0;
            const T* x01 = a.in + (int64_t)n01 * KB + b0;
            const T* x11 = a.in + (int64_t)(n01 + a.n_phi) * KB + b0;
            if (vec && nb == BC) {
                constexpr int Q = BC / VW > 0 ? BC / VW : 1;
                V* zsv = reinterpret_cast<V*>(zs);
                const int n_items = nwin * Q;
                for (int base = 0; base < n_items; base += 64) {
                    V v[2][4];
                    bool okv[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int o = base + lane + 32 * u;
                        const int kk = o / Q, q = o - kk * Q;
                        const int k = k_lo + kk;
                        okv[u] = o < n_items && k >= 0 && k < a.K;
                        if (okv[u]) {
                            const int64_t off = (int64_t)k * a.B + VW * q;
                            v[u][0] = __ldg(reinterpret_cast<const V*>(x00 + off));
                            v[u][1] = __ldg(reinterpret_cast<const V*>(x10 + off));
                            v[u][2] = __ldg(reinterpret_cast<const V*>(x01 + off));
                            v[u][3] = __ldg(reinterpret_cast<const V*>(x11 + off));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int o = base + lane + 32 * u;
                        if (o < n_items) {
                            V z;
                            T* zc = comps<T>(z);
#pragma unroll
                            for (int c = 0; c < VW; ++c) {
                                zc[c] = okv[u] ? w[0] * comps<T>(v[u][0])[c] + w[1] * comps<T>(v[u][1])[c] +
                                                     w[2] * comps<T>(v[u][2])[c] + w[3] * comps<T>(v[u][3])[c]
                                               : T(0);
                            }
                            zsv[o] = z;
                        }
                    }
                }
            } else {
                for (int o = lane; o < nwin * BC; o += 32) {
                    const int kk = o / BC, bb = o - kk * BC;
                    const int k = k_lo + kk;
                    T z = T(0);
                    if (k >= 0 && k < a.K && bb < nb) {
                        const int64_t off = (int64_t)k * a.B + bb;
                        z = w[0] * x00[off] + w[1] * x10[off] + w[2] * x01[off] + w[3] * x11[off];
                    }
                    zs[o] = z;
                }
            }
            __syncwarp();
            int64_t U = U0 - (int64_t)(f_begin + lane) * a.D;
            const int64_t dU = (int64_t)32 * a.D;
#pragma unroll
            for (int j = 0; j < FPL; ++j) {
                const int f = f_begin + lane + 32 * j;
                if (f < f_end) {
                    const int k0 = (int)(U >> kFracBits);
                    const T fr = frac_of<T>(U, f, a.D, F64);
                    const T g = T(1) - fr;
                    const T* z0 = zs + (k0 - k_lo) * BC;
                    if constexpr (BC >= VW) {
#pragma unroll
                        for (int q = 0; q < BC / VW; ++q) {
                            const V p0 = reinterpret_cast<const V*>(z0)[q];
                            const V p1 = reinterpret_cast<const V*>(z0 + BC)[q];
#pragma unroll
                            for (int c = 0; c < VW; ++c)
                                acc[j][VW * q + c] += g * comps<T>(p0)[c] + fr * comps<T>(p1)[c];
                        }
                    } else {
#pragma unroll
                        for (int b = 0; b < BC; ++b) acc[j][b] += g * z0[b] + fr * z0[BC + b];
                    }
                }
                U -= dU;
            }
            __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < FPL; ++j) {
            const int f = f_begin + lane + 32 * j;
            if (f >= f_end) continue;
            T* yo = a.out + ((int64_t)row_out * a.Tn + f) * a.B + b0;
            if (vec && nb == BC) {
#pragma unroll
                for (int q = 0; q < BC / VW; ++q) {
                    V o;
#pragma unroll
                    for (int c = 0; c < VW; ++c) comps<T>(o)[c] = acc[j][VW * q + c];
                    reinterpret_cast<V*>(yo)[q] = o;
                }
            } else {
#pragma unroll
                for (int b = 0; b < BC; ++b)
                    if (b < nb) yo[b] = acc[j][b];
            }
        }
    }
}

// Adjoint phase 1, fast path: lane per hat within a group of 32 hats; the
// frames feeding the group are staged once in shared memory and each lane
// accumulates all BC batch entries of its hat.
constexpr int kAdj3Warps = 4;

// Swizzled staging layout: the 16-byte chunk index of (frame f, chunk q) has
// its low three bits XORed with (f / P) mod 8, P = frames per hat step, so
// the lanes of a warp (one hat each, hats P frames apart) read eight distinct
// bank groups.
__device__ __forceinline__ int swz(int f, int q, int Q, int pshift) {
    const int idx = f * Q + q;
    return idx ^ ((f >> pshift) & 7);
}

template <typename T, int BC>
__global__ void __launch_bounds__(kAdj3Warps * 32)
adj_time3_kernel(const ApplyArgs<T> a) {
    using V = typename Vec16<T>::type;
    constexpr int VW = Vec16<T>::W;
    extern __shared__ __align__(16) unsigned char smem_a3_raw[];
    T* ys = reinterpret_cast<T*>(smem_a3_raw) + (threadIdx.x >> 5) * (a.zwin * BC);
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * kAdj3Warps + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * kAdj3Warps;
    const bool vec = (BC >= VW) && a.vec4 && (a.Bc == BC);
    constexpr int Q = BC / VW > 0 ? BC / VW : 1;
    const int P = a.FC;  // log2 of frames per hat step, used only for the swizzle
    const float invD = 1.0f / (float)a.D;
    const int32_t D32 = (int32_t)a.D;  // D <= 2^24
    for (int64_t e = warp_global; e < a.n_tasks; e += n_warps) {
        const int row_out = seg_out_row(a.seg, a.ray_row[e]);
        if (row_out < 0) {
            // rays outside the arm contribute nothing: their zhat rows are zero
            T* zo = a.zhat + (int64_t)e * a.K * a.Bc;
            for (int o = lane; o < a.K * a.Bc; o += 32) zo[o] = T(0);
            continue;
        }
        const int64_t U0 = (int64_t)a.K0[e] * kFracOne + (int64_t)a.F0[e];
        const double F64 = exact_frac(a, (int)e);
        const T* yrow = a.in + (int64_t)row_out * a.Tn * a.B;
        for (int kg0 = 0; kg0 < a.K; kg0 += 32) {
            const int kg1 = min(kg0 + 31, a.K - 1);
            // frames with (kg0 - 1) 2^24 <= U(f) < (kg1 + 1) 2^24, found from a float
            // estimate corrected by exact integer tests
            const int64_t hiX = (int64_t)(kg1 + 1) * kFracOne;
            const int64_t loX = (int64_t)(kg0 - 1) * kFracOne;
            int fA = (int)fminf(fmaxf(floorf((float)(U0 - hiX) * invD) - 1.0f, 0.0f), (float)a.Tn);
            while (fA < a.Tn && U0 - (int64_t)fA * a.D >= hiX) ++fA;
            int fB = (int)fminf(fmaxf(floorf((float)(U0 - loX) * invD) + 1.0f, -1.0f),
                                (float)(a.Tn - 1));
            while (fB >= 0 && U0 - (int64_t)fB * a.D < loX) --fB;
            const int nfr = fB >= fA ? fB - fA + 1 : 0;
            if (vec) {
                V* ysv = reinterpret_cast<V*>(ys);
                for (int o = lane; o < nfr * Q; o += 32) {
                    const int fl = o / Q, q = o - fl * Q;
                    ysv[swz(fl, q, Q, P)] =
                        __ldg(reinterpret_cast<const V*>(yrow + (int64_t)(fA + fl) * a.B) + q);
                }
            } else {
                for (int o = lane; o < nfr * BC; o += 32) {
                    const int fl = o / BC, bb = o - fl * BC;
                    ys[o] = bb < a.Bc ? yrow[(int64_t)(fA + fl) * a.B + bb] : T(0);
                }
            }
            __syncwarp();
            const int k = kg0 + lane;
            if (k <= kg1) {
                T acc[BC];
#pragma unroll
                for (int b = 0; b < BC; ++b) acc[b] = T(0);
                // frames with |U(f) - k 2^24| < 2^24 (hat k's support); in that
                // window Ur = U(f) - k 2^24 fits 32 bits and the hat weight is
                // 1 - |Ur| 2^-24 exactly (FP32); FP64 uses the exact fraction
                const int64_t hi_excl = (int64_t)(k + 1) * kFracOne;
                const float est = (float)(U0 - hi_excl) * invD;
                int f = (int)fminf(fmaxf(floorf(est) - 1.0f, (float)fA), (float)(fB + 1));
                int64_t U = U0 - (int64_t)f * a.D;
                while (f <= fB && U >= hi_excl) { ++f; U -= a.D; }
                int32_t Ur = (int32_t)(U - (int64_t)k * kFracOne);  // in [-2^24, 2^24) once f <= fB
                for (; f <= fB && Ur > -kFracOne; ++f, Ur -= D32) {
                    T hw;
                    if constexpr (sizeof(T) == 4) {
                        hw = 1.0f - (float)abs(Ur) * (1.0f / (float)kFracOne);
                    } else {
                        const int64_t Uf = (int64_t)k * kFracOne + Ur;
                        const int k0 = (int)(Uf >> kFracBits);
                        const T fr = frac_of<T>(Uf, f, a.D, F64);
                        hw = (k0 == k) ? T(1) - fr : fr;
                    }
                    if (vec) {
                        const V* ysv = reinterpret_cast<const V*>(ys);
#pragma unroll
                        for (int q = 0; q < Q; ++q) {
                            const V t = ysv[swz(f - fA, q, Q, P)];
#pragma unroll
                            for (int c = 0; c < VW; ++c) acc[VW * q + c] += hw * comps<T>(t)[c];
                        }
                    } else {
                        const T* yv = ys + (f - fA) * BC;
#pragma unroll
                        for (int b = 0; b < BC; ++b) acc[b] += hw * yv[b];
                    }
                }
                T* zo = a.zhat + ((int64_t)e * a.K + k) * a.Bc;
                if (vec) {
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        V o;
#pragma unroll
                        for (int c = 0; c < VW; ++c) comps<T>(o)[c] = acc[VW * q + c];
                        reinterpret_cast<V*>(zo)[q] = o;
                    }
                } else {
#pragma unroll
                    for (int b = 0; b < BC; ++b)
                        if (b < a.Bc) zo[b] = acc[b];
                }
            }
            __syncwarp();
        }
    }
}

// Adjoint phase 2, fast path: lanes over (hat, batch) of one node, nodes in
// descending-load order; the incidence loop is unrolled by 4 so that four
// zhat rows are in flight.
template <typename T>
__device__ __forceinline__ T corner_coef(const ApplyArgs<T>& a, int code);
template <>
__device__ __forceinline__ float corner_coef<float>(const ApplyArgs<float>& a, int code) {
    return reinterpret_cast<const float*>(a.W)[code];  // W[e] component c = element 4e + c
}
template <>
__device__ __forceinline__ double corner_coef<double>(const ApplyArgs<double>& a, int code) {
    return a.W64[code];
}

template <typename T, int BC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
adj_space3_kernel(const ApplyArgs<T> a) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t task = warp_global; task < a.n_tasks; task += n_warps) {
        const int kchunk = (int)(task % a.n_kchunk);
        const int node = a.node_order ? a.node_order[task / a.n_kchunk] : (int)(task / a.n_kchunk);
        const int k_begin = kchunk * a.KC;
        T acc[kAdjOutPerLane];
#pragma unroll
        for (int j = 0; j < kAdjOutPerLane; ++j) acc[j] = T(0);
        int off[kAdjOutPerLane];
        bool live[kAdjOutPerLane];
#pragma unroll
        for (int j = 0; j < kAdjOutPerLane; ++j) {
            const int o = lane + 32 * j;
            const int kk = o / BC, bb = o - kk * BC;
            const int k = k_begin + kk;
            live[j] = kk < a.KC && k < a.K && bb < a.Bc;
            off[j] = k * a.Bc + bb;
        }
        const int i_begin = a.node_ptr[node], i_end = a.node_ptr[node + 1];
        int ii = i_begin;
        // incidence codes of the next group of 4 are loaded before the current
        // group's zhat rows are consumed (two loads levels in flight)
        int nxt[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) nxt[u] = (ii + u < i_end) ? a.inc[ii + u] : 0;
        for (; ii + 4 <= i_end; ii += 4) {
            int code[4];
            T coef[4];
            const T* zr[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) code[u] = nxt[u];
#pragma unroll
            for (int u = 0; u < 4; ++u) nxt[u] = (ii + 4 + u < i_end) ? a.inc[ii + 4 + u] : 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                coef[u] = corner_coef(a, code[u]);
                zr[u] = a.zhat + (int64_t)(code[u] >> 2) * a.K * a.Bc;
            }
#pragma unroll
            for (int j = 0; j < kAdjOutPerLane; ++j) {
                if (!live[j]) continue;
                const T v0 = zr[0][off[j]], v1 = zr[1][off[j]], v2 = zr[2][off[j]], v3 = zr[3][off[j]];
                acc[j] += coef[0] * v0;
                acc[j] += coef[1] * v1;
                acc[j] += coef[2] * v2;
                acc[j] += coef[3] * v3;
            }
        }
        for (; ii < i_end; ++ii) {
            const int code = a.inc[ii];
            const T coef = corner_coef(a, code);
            const T* zr = a.zhat + (int64_t)(code >> 2) * a.K * a.Bc;
#pragma unroll
            for (int j = 0; j < kAdjOutPerLane; ++j)
                if (live[j]) acc[j] += coef * zr[off[j]];
        }
#pragma unroll
        for (int j = 0; j < kAdjOutPerLane; ++j) {
            if (!live[j]) continue;
            const int o = lane + 32 * j;
            const int kk = o / BC, bb = o - kk * BC;
            a.out[((int64_t)node * a.K + k_begin + kk) * a.B + bb] = acc[j];
        }
    }
}

static int pick_bc(int B) {
    int bc = 1;
    while (bc < B && bc < 32) bc <<= 1;
    return bc;
}

static int grid_for(int64_t n_tasks) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n_tasks + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int64_t cap = (int64_t)sms * 16;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <typename T>
static ApplyArgs<T> base_args(const rtt_op_s* op, const T* in, T* out, int B, const ArmSeg& seg) {
    ApplyArgs<T> a{};
    a.row_ptr = op->row_ptr;
    a.ray_row = op->ray_row;
    a.row_order = op->row_order;
    a.node00 = op->node00;
    a.node01 = op->node01;
    a.W = op->W;
    a.W64 = op->W64;
    a.K0 = op->K0;
    a.F0 = op->F0;
    a.F64 = op->F64;
    a.node_ptr = op->node_ptr;
    a.inc = op->inc;
    a.in = in;
    a.out = out;
    a.B = B;
    a.K = op->time.n_hats;
    a.Tn = op->time.n_frames;
    a.n_phi = op->grid.n_phi;
    a.n_nodes = op->n_nodes;
    a.D = op->frame_D;
    a.delta = op->delta;
    a.seg = seg;
    a.seg_rows_all = (int)op->n_rows;
    a.node_order = op->node_order;
    return a;
}

template <typename T, int BC>
static cudaError_t launch_fwd3_bc(ApplyArgs<T> a, cudaStream_t st) {
    constexpr int FPL = BC >= 32 ? 1 : 32 / BC;
    a.FC = 32 * FPL;
    a.vec4 = (a.B % Vec16<T>::W == 0) ? 1 : 0;
    a.zwin = (int)ceil((a.FC - 1) * a.delta) + 3;
    a.n_fchunk = (a.Tn + a.FC - 1) / a.FC;
    a.n_bchunk = (a.B + BC - 1) / BC;
    a.n_tasks = (int64_t)a.seg.total * a.n_fchunk * a.n_bchunk;
    if (a.n_tasks == 0) return cudaSuccess;
    const size_t smem = (size_t)kWarpsPerBlock * a.zwin * BC * sizeof(T);
    if (smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(fwd3_kernel<T, BC>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    fwd3_kernel<T, BC><<<grid_for(a.n_tasks), kWarpsPerBlock * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_forward(const rtt_op_s* op, const T* x, T* y, int B, const ArmSeg& seg,
                           cudaStream_t st) {
    ApplyArgs<T> a = base_args<T>(op, x, y, B, seg);
    switch (pick_bc(B)) {
        case 1: return launch_fwd3_bc<T, 1>(a, st);
        case 2: return launch_fwd3_bc<T, 2>(a, st);
        case 4: return launch_fwd3_bc<T, 4>(a, st);
        case 8: return launch_fwd3_bc<T, 8>(a, st);
        case 16: return launch_fwd3_bc<T, 16>(a, st);
        default: return launch_fwd3_bc<T, 32>(a, st);
    }
}

// Adjoint: fast phase 1 when the frames of a 32-hat group fit the staging
// buffer, otherwise the general per-(hat, batch) kernel; then the gather.
template <typename T, int BC>
static cudaError_t launch_adj3_bc(ApplyArgs<T> a, cudaStream_t st) {
    // staged frames per 32-hat group, rounded so the swizzle stays in bounds
    int ywin = (int)ceil(33.0 / a.delta) + 2;
    ywin = (ywin + 7) & ~7;
    const size_t smem = (size_t)kAdj3Warps * ywin * BC * sizeof(T);
    cudaError_t e = cudaSuccess;
    if (a.seg.total > 0) {
        if (smem <= 96 * 1024) {
            ApplyArgs<T> t = a;
            t.zwin = ywin;
            {
                // log2 of the frames per hat step (swizzle key only)
                int ps = 0;
                while ((2 << ps) <= (int)floor(1.0 / a.delta + 0.5)) ++ps;
                t.FC = ps;
            }
            t.vec4 = (a.B % Vec16<T>::W == 0) ? 1 : 0;
            t.n_tasks = a.n_rays_total;
            if (smem > 48 * 1024) {
                e = cudaFuncSetAttribute(adj_time3_kernel<T, BC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
            const int64_t want = (t.n_tasks + kAdj3Warps - 1) / kAdj3Warps;
            int dev = 0, sms = 148;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int grid = (int)(want < (int64_t)sms * 32 ? (want > 0 ? want : 1) : (int64_t)sms * 32);
            adj_time3_kernel<T, BC><<<grid, kAdj3Warps * 32, smem, st>>>(t);
            e = cudaGetLastError();
        } else {
            ApplyArgs<T> t = a;
            t.KC = kAdjOutPerLane * 32 / BC;
            t.n_kchunk = (a.K + t.KC - 1) / t.KC;
            t.n_bchunk = 1;
            t.n_tasks = a.n_rays_total * t.n_kchunk;
            adj_time_kernel<T, BC><<<grid_for(t.n_tasks), kWarpsPerBlock * 32, 0, st>>>(t);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
    }
    a.KC = kAdjOutPerLane * 32 / BC;
    a.n_kchunk = (a.K + a.KC - 1) / a.KC;
    a.n_bchunk = 1;
    a.n_tasks = (int64_t)a.n_nodes * a.n_kchunk;
    if (a.n_tasks == 0) return cudaSuccess;
    adj_space3_kernel<T, BC><<<grid_for(a.n_tasks), kWarpsPerBlock * 32, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_fused(const rtt_op_s* op, const float* y, float* x, int B, int b_first,
                                 int Bc, const ArmSeg& seg, float* partial, cudaStream_t st);

template <typename T>
cudaError_t launch_adjoint(const rtt_op_s* op, const T* y, T* x, int B, const ArmSeg& seg,
                           T* zhat, cudaStream_t st) {
    if (seg.total == 0)  // no data rows in the arm: A^T y = 0
        return cudaMemsetAsync(x, 0, (size_t)op->n_nodes * op->time.n_hats * B * sizeof(T), st);
    // batch chunks of at most 32 entries share the zhat scratch [E][K][32]
    for (int b_first = 0; b_first < B; b_first += 32) {
        const int Bc = B - b_first < 32 ? B - b_first : 32;
        ApplyArgs<T> a = base_args<T>(op, y + b_first, x + b_first, B, seg);
        a.zhat = zhat;
        a.Bc = Bc;
        a.n_rays_total = op->n_rays;
        cudaError_t e;
        if constexpr (sizeof(T) == 4) {
            if (op->use_fused_adjoint && (op->fpartial || op->n_partial_slots == 0)) {
                e = launch_adjoint_fused(op, y, x, B, b_first, Bc, seg, (float*)op->fpartial, st);
                if (e == cudaSuccess) continue;
                if (e != cudaErrorNotSupported) return e;
                cudaGetLastError();  // clear the "not supported" marker
            }
            switch (pick_bc(Bc)) {
                case 1: e = launch_adj3_bc<T, 1>(a, st); break;
                case 2: e = launch_adj3_bc<T, 2>(a, st); break;
                case 4: e = launch_adj3_bc<T, 4>(a, st); break;
                case 8: e = launch_adj3_bc<T, 8>(a, st); break;
                case 16: e = launch_adj3_bc<T, 16>(a, st); break;
                default: e = launch_adj3_bc<T, 32>(a, st); break;
            }
        } else {
            switch (pick_bc(Bc)) {
                case 1: e = launch_adj3_bc<T, 1>(a, st); break;
                case 2: e = launch_adj3_bc<T, 2>(a, st); break;
                case 4: e = launch_adj3_bc<T, 4>(a, st); break;
                case 8: e = launch_adj3_bc<T, 8>(a, st); break;
                case 16: e = launch_adj3_bc<T, 16>(a, st); break;
                default: e = launch_adj3_bc<T, 32>(a, st); break;
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t launch_forward<float>(const rtt_op_s*, const float*, float*, int, const ArmSeg&,
                                           cudaStream_t);
template cudaError_t launch_forward<double>(const rtt_op_s*, const double*, double*, int,
                                            const ArmSeg&, cudaStream_t);
template cudaError_t launch_adjoint<float>(const rtt_op_s*, const float*, float*, int, const ArmSeg&,
                                           float*, cudaStream_t);
template cudaError_t launch_adjoint<double>(const rtt_op_s*, const double*, double*, int,
                                            const ArmSeg&, double*, cudaStream_t);

}  // namespace rtt
