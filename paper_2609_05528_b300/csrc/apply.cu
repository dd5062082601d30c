// Forward operator A (Sec. 3.1 Eq. 2-3, Eq. 16, Eq. 47); the adjoint is in
// adjoint.cu.
//
// One warp per (row, frame chunk, batch chunk): for each ray e of the row,
// the spatially interpolated history z_e[k][b] = sum_c W_{e,c} x[node_c][k][b]
// is staged in shared memory for the hats the frame chunk can touch, then
// every output sample adds (1 - fr) z_e[k0] + fr z_e[k0 + 1] with the exact
// integer hat index k0 and 24-bit fraction fr of that (ray, frame).  y is
// written once, coalesced.
#include <cuda.h>  // CUtensorMap and its enums (types only; no driver-library link)
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "kern_common.cuh"

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
    const uint2* W16;  // BF16 copy of W (weights of BF16 precision), or null
    const double* W64;
    const int32_t* K0;
    const int32_t* F0;
    const float4* ray_rec;   // per ray (K0, F0, node00, node01 as int bits), W; or null
    const double* F64;
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
    int64_t n_rays_total;
    int seg_rows_all;  // total rows of the operator (all orders)
    int* status;                // device status word (bit 0: a bounded wait timed out)
    const int32_t* row_sched;   // rows in source-cell order within each order, or null
    int Bcols;                  // columns of this launch (0: all B), the periodic forward
    int hs32;                   // hat steps per 32 frames when a whole number, else 0
    int n_fchunk, n_bchunk, n_kchunk;
    int64_t n_tasks;
};

template <typename T>
__device__ __forceinline__ void load_w(const ApplyArgs<T>& a, int e, T w[4]);

template <>
__device__ __forceinline__ void load_w<float>(const ApplyArgs<float>& a, int e, float w[4]) {
    const float4 v = corner_weights(a.W, a.W16, e);
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

// output row and input row of the t-th task row of the arm: the natural
// (order, pixel) order, or the source-cell order of the operator's row
// schedule (a permutation within each order, so the arm's rows stay a union
// of whole order blocks)
template <typename T>
__device__ __forceinline__ void task_row(const ApplyArgs<T>& a, int t, int& row_out, int& row) {
    if (a.row_sched) {
        row = a.row_sched[seg_in_row(a.seg, t)];
        row_out = seg_out_row(a.seg, row);
    } else {
        row_out = t;
        row = seg_in_row(a.seg, t);
    }
}

// spatial interpolation w0 v0 + w1 v1 + w2 v2 + w3 v3
template <typename T>
__device__ __forceinline__ T interp4(T w0, T v0, T w1, T v1, T w2, T v2, T w3, T v3) {
    return fmac(w3, v3, fmac(w2, v2, fmac(w1, v1, w0 * v0)));
}
// temporal interpolation acc + g z0 + fr z1
template <typename T>
__device__ __forceinline__ T hat2(T acc, T g, T z0, T fr, T z1) {
    return fmac(fr, z1, fmac(g, z0, acc));
}

constexpr int kWarpsPerBlock = 8;

// Grid-stride walk over (output row, frame chunk, batch chunk) tasks, batch
// chunk fastest (task = (row nf + f) nb + b).  The first task and the stride
// are split into those digits once; each step adds the stride's digits with
// carries, so no task index is divided inside the loop.
struct TaskWalk {
    int b, f, r;     // current task
    int db, df, dr;  // grid stride in the same digits
    int nb, nf;
    __device__ __forceinline__ TaskWalk(int64_t start, int64_t stride, int nb_, int nf_)
        : nb(nb_), nf(nf_) {
        b = (int)(start % nb);
        int64_t q = start / nb;
        f = (int)(q % nf);
        r = (int)(q / nf);
        db = (int)(stride % nb);
        q = stride / nb;
        df = (int)(q % nf);
        dr = (int)(q / nf);
    }
    __device__ __forceinline__ void next() {
        b += db;
        int c = b >= nb ? 1 : 0;
        b -= c * nb;
        f += df + c;
        c = f >= nf ? 1 : 0;
        f -= c * nf;
        r += dr + c;
    }
};

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

// FPL frames per lane (32 FPL per task); SU staging items in flight per lane
// and pass.  Fewer accumulators per lane (BC FPL <= 16) or one item in
// flight (SU = 1) allow three resident CTAs per SM.
template <typename T, int BC, int FPL, int SU = 2>
__global__ void __launch_bounds__(kWarpsPerBlock * 32,
                                  (sizeof(T) == 8 || BC >= 32) ? 1
                                                               : ((BC * FPL <= 16 || SU == 1) ? 3 : 2))
fwd3_kernel(const ApplyArgs<T> a) {
    using V = typename Vec16<T>::type;
    constexpr int VW = Vec16<T>::W;
    constexpr int FC = 32 * FPL;  // frames per task
    extern __shared__ __align__(16) unsigned char smem3_raw[];
    T* zs = reinterpret_cast<T*>(smem3_raw) + (threadIdx.x >> 5) * (a.zwin * BC);
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * kWarpsPerBlock;
    const bool vec = (BC >= VW) && a.vec4;
    for (TaskWalk tw(warp_global, n_warps, a.n_bchunk, a.n_fchunk); tw.r < a.seg.total; tw.next()) {
        const int bchunk = tw.b;
        const int fchunk = tw.f;
        int row_out, row;
        task_row(a, tw.r, row_out, row);
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
                for (int base = 0; base < n_items; base += 32 * SU) {
                    V v[SU][4];
                    bool okv[SU];
#pragma unroll
                    for (int u = 0; u < SU; ++u) {
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
                    for (int u = 0; u < SU; ++u) {
                        const int o = base + lane + 32 * u;
                        if (o < n_items) {
                            V z;
                            T* zc = comps<T>(z);
                            if constexpr (sizeof(T) == 4) {
                                // packed FP32 pairs, the operations of interp4 per component
#pragma unroll
                                for (int c = 0; c < VW; c += 2) {
                                    float2 r = __fmul2_rn(make_float2(w[0], w[0]),
                                                          make_float2(comps<T>(v[u][0])[c], comps<T>(v[u][0])[c + 1]));
                                    r = __ffma2_rn(make_float2(w[1], w[1]),
                                                   make_float2(comps<T>(v[u][1])[c], comps<T>(v[u][1])[c + 1]), r);
                                    r = __ffma2_rn(make_float2(w[2], w[2]),
                                                   make_float2(comps<T>(v[u][2])[c], comps<T>(v[u][2])[c + 1]), r);
                                    r = __ffma2_rn(make_float2(w[3], w[3]),
                                                   make_float2(comps<T>(v[u][3])[c], comps<T>(v[u][3])[c + 1]), r);
                                    zc[c] = okv[u] ? r.x : T(0);
                                    zc[c + 1] = okv[u] ? r.y : T(0);
                                }
                            } else {
#pragma unroll
                                for (int c = 0; c < VW; ++c) {
                                    zc[c] = okv[u] ? interp4(w[0], comps<T>(v[u][0])[c], w[1],
                                                             comps<T>(v[u][1])[c], w[2], comps<T>(v[u][2])[c],
                                                             w[3], comps<T>(v[u][3])[c])
                                                   : T(0);
                                }
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
                        z = interp4(w[0], x00[off], w[1], x10[off], w[2], x01[off], w[3], x11[off]);
                    }
                    zs[o] = z;
                }
            }
            __syncwarp();
            // (1 - fr) z[k0] + fr z[k0 + 1] for frame j of this lane
            auto add_frame = [&](int j, int k0, T fr) {
                const T g = T(1) - fr;
                const T* z0 = zs + (k0 - k_lo) * BC;
                if constexpr (BC >= VW) {
#pragma unroll
                    for (int q = 0; q < BC / VW; ++q) {
                        const V p0 = reinterpret_cast<const V*>(z0)[q];
                        const V p1 = reinterpret_cast<const V*>(z0 + BC)[q];
                        if constexpr (sizeof(T) == 4) {
                            // packed FP32 pairs: per component the fused
                            // multiply-adds of hat2, in the same order
                            const float2 g2 = make_float2(g, g), f2 = make_float2(fr, fr);
#pragma unroll
                            for (int c = 0; c < VW; c += 2) {
                                float2 s2 = make_float2(acc[j][VW * q + c], acc[j][VW * q + c + 1]);
                                s2 = __ffma2_rn(g2, make_float2(comps<T>(p0)[c], comps<T>(p0)[c + 1]), s2);
                                s2 = __ffma2_rn(f2, make_float2(comps<T>(p1)[c], comps<T>(p1)[c + 1]), s2);
                                acc[j][VW * q + c] = s2.x;
                                acc[j][VW * q + c + 1] = s2.y;
                            }
                        } else {
#pragma unroll
                            for (int c = 0; c < VW; ++c)
                                acc[j][VW * q + c] =
                                    hat2(acc[j][VW * q + c], g, comps<T>(p0)[c], fr, comps<T>(p1)[c]);
                        }
                    }
                } else {
#pragma unroll
                    for (int b = 0; b < BC; ++b) acc[j][b] = hat2(acc[j][b], g, z0[b], fr, z0[BC + b]);
                }
            };
            const int64_t U1 = U0 - (int64_t)(f_begin + lane) * a.D;
            if (a.hs32 > 0) {
                // 32 frames are hs32 whole hat steps: a lane's frames share the
                // hat fraction and step down hs32 hats from one to the next
                // (the same k0 and fraction as the per-frame computation)
                const int k00 = (int)(U1 >> kFracBits);
                const T fr0 = frac_of<T>(U1, f_begin + lane, a.D, F64);
#pragma unroll
                for (int j = 0; j < FPL; ++j)
                    if (f_begin + lane + 32 * j < f_end) add_frame(j, k00 - j * a.hs32, fr0);
            } else {
                int64_t U = U1;
                const int64_t dU = (int64_t)32 * a.D;
#pragma unroll
                for (int j = 0; j < FPL; ++j) {
                    const int f = f_begin + lane + 32 * j;
                    if (f < f_end) add_frame(j, (int)(U >> kFracBits), frac_of<T>(U, f, a.D, F64));
                    U -= dU;
                }
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

// Forward when a frame step is exactly 1/P of a hat step (P an integer,
// FP32).  Lane l owns the P consecutive frames f_c + P l + j (j < P) of the
// task's chunk.  For every ray those frames lie between the lane's own hat
// k_l = floor(u(f_c)) - l and its neighbours k_l +- 1, with the same
// fractional phase on every lane, so each lane forms the spatially
// interpolated history z of its own hat only (4 corner loads) and takes the
// neighbours' z by warp shuffles; lanes 0 and 31 also form the two hats just
// outside the warp.  No shared memory and no per-frame index arithmetic
// beyond one comparison; the hat index, fraction and summation order per
// output are those of fwd3_kernel.
template <int BC, int P>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 2)
fwd4_kernel(const ApplyArgs<float> a) {
    constexpr int Q = BC >= 4 ? BC / 4 : 1;
    constexpr int FC = 32 * P;
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * kWarpsPerBlock;
    const int32_t D32 = (int32_t)a.D;  // 2^24 / P
    const int64_t KB = (int64_t)a.K * a.B;
    for (int64_t task = warp_global; task < a.n_tasks; task += n_warps) {
        const int bchunk = (int)(task % a.n_bchunk);
        const int64_t t2 = task / a.n_bchunk;
        const int fchunk = (int)(t2 % a.n_fchunk);
        int row_out, row;
        task_row(a, (int)(t2 / a.n_fchunk), row_out, row);
        const int f_c = fchunk * FC;
        const int b0 = bchunk * BC;
        const int nb = min(BC, a.B - b0);
        const bool vec = (BC >= 4) && a.vec4 && nb == BC;
        float acc[P][BC];
#pragma unroll
        for (int j = 0; j < P; ++j)
#pragma unroll
            for (int b = 0; b < BC; ++b) acc[j][b] = 0.0f;
        const int e_begin = a.row_ptr[row], e_end = a.row_ptr[row + 1];
        for (int e = e_begin; e < e_end; ++e) {
            const int64_t Ub = (int64_t)a.K0[e] * kFracOne + (int64_t)a.F0[e] - (int64_t)f_c * a.D;
            const int k_top = (int)(Ub >> kFracBits);         // own hat of lane 0
            const int32_t phase = (int32_t)(Ub & kFracMask);  // same on every lane
            const int k_own = k_top - lane;
            // lanes 0 and 31 also need the hats k_top + 1 and k_top - 32
            const int k_ext = lane == 0 ? k_top + 1 : k_top - 32;
            const bool ext = lane == 0 || lane == 31;
            const float4 wv = corner_weights(a.W, a.W16, e);
            const int n00 = a.node00[e], n01 = a.node01[e];
            const float* x00 = a.in + (int64_t)n00 * KB + b0;
            const float* x10 = a.in + (int64_t)(n00 + a.n_phi) * KB + b0;
            const float* x01 = a.in + (int64_t)n01 * KB + b0;
            const float* x11 = a.in + (int64_t)(n01 + a.n_phi) * KB + b0;
            float z[BC], zx[BC];
            const bool own_ok = k_own >= 0 && k_own < a.K;
            const bool ext_ok = ext && k_ext >= 0 && k_ext < a.K;
            if (vec) {
                float4 v[2][Q][4];
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int64_t o0 = (int64_t)k_own * a.B + 4 * q, o1 = (int64_t)k_ext * a.B + 4 * q;
                    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
                    v[0][q][0] = own_ok ? __ldg(reinterpret_cast<const float4*>(x00 + o0)) : zero;
                    v[0][q][1] = own_ok ? __ldg(reinterpret_cast<const float4*>(x10 + o0)) : zero;
                    v[0][q][2] = own_ok ? __ldg(reinterpret_cast<const float4*>(x01 + o0)) : zero;
                    v[0][q][3] = own_ok ? __ldg(reinterpret_cast<const float4*>(x11 + o0)) : zero;
                    v[1][q][0] = ext_ok ? __ldg(reinterpret_cast<const float4*>(x00 + o1)) : zero;
                    v[1][q][1] = ext_ok ? __ldg(reinterpret_cast<const float4*>(x10 + o1)) : zero;
                    v[1][q][2] = ext_ok ? __ldg(reinterpret_cast<const float4*>(x01 + o1)) : zero;
                    v[1][q][3] = ext_ok ? __ldg(reinterpret_cast<const float4*>(x11 + o1)) : zero;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        const float* c0 = reinterpret_cast<const float*>(&v[h][q][0]);
                        const float* c1 = reinterpret_cast<const float*>(&v[h][q][1]);
                        const float* c2 = reinterpret_cast<const float*>(&v[h][q][2]);
                        const float* c3 = reinterpret_cast<const float*>(&v[h][q][3]);
                        float* zz = h == 0 ? z : zx;
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            zz[4 * q + c] = interp4(wv.x, c0[c], wv.y, c1[c], wv.z, c2[c], wv.w, c3[c]);
                    }
            } else {
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    z[b] = 0.0f;
                    zx[b] = 0.0f;
                    if (b < nb) {
                        if (own_ok) {
                            const int64_t o = (int64_t)k_own * a.B + b;
                            z[b] = interp4(wv.x, x00[o], wv.y, x10[o], wv.z, x01[o], wv.w, x11[o]);
                        }
                        if (ext_ok) {
                            const int64_t o = (int64_t)k_ext * a.B + b;
                            zx[b] = interp4(wv.x, x00[o], wv.y, x10[o], wv.z, x01[o], wv.w, x11[o]);
                        }
                    }
                }
            }
            // z of hat k_own + 1 (lane l - 1) and k_own - 1 (lane l + 1)
            float zu[BC], zd[BC];
#pragma unroll
            for (int b = 0; b < BC; ++b) {
                const float up = __shfl_up_sync(0xffffffffu, z[b], 1);
                const float dn = __shfl_down_sync(0xffffffffu, z[b], 1);
                zu[b] = lane == 0 ? zx[b] : up;
                zd[b] = lane == 31 ? zx[b] : dn;
            }
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int32_t Uj = phase - j * D32;  // U(f) - k_own 2^24, in [-2^24, 2^24)
                if (Uj >= 0) {  // hat base k_own
                    const float fr = (float)Uj * (1.0f / (float)kFracOne);
                    const float g = 1.0f - fr;
#pragma unroll
                    for (int b = 0; b < BC; ++b) acc[j][b] = hat2(acc[j][b], g, z[b], fr, zu[b]);
                } else {  // hat base k_own - 1
                    const float fr = (float)(Uj + kFracOne) * (1.0f / (float)kFracOne);
                    const float g = 1.0f - fr;
#pragma unroll
                    for (int b = 0; b < BC; ++b) acc[j][b] = hat2(acc[j][b], g, zd[b], fr, z[b]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int f = f_c + P * lane + j;
            if (f >= a.Tn) continue;
            float* yo = a.out + ((int64_t)row_out * a.Tn + f) * a.B + b0;
            if (vec) {
#pragma unroll
                for (int q = 0; q < Q; ++q)
                    reinterpret_cast<float4*>(yo)[q] = make_float4(acc[j][4 * q], acc[j][4 * q + 1],
                                                                   acc[j][4 * q + 2], acc[j][4 * q + 3]);
            } else {
#pragma unroll
                for (int b = 0; b < BC; ++b)
                    if (b < nb) yo[b] = acc[j][b];
            }
        }
    }
}

// Forward with the four corner slabs of x staged by the tensor memory
// accelerator.  Same tasks, hat windows, interpolation and accumulation order
// as fwd3_kernel<float, BC, FPL> (hence the same bits); what changes is how
// x reaches shared memory: per ray, four 3D tiled copies (one per corner
// node: BC batch entries x zwin hats starting at the window's first hat,
// out-of-range hats zero-filled by the copy) land in a double buffer while
// the previous ray is contracted, so the loads of ray e + 1 overlap the
// arithmetic of ray e.  Waits are bounded as in adj_time5_kernel.
template <int BC, int FPL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, BC * FPL <= 16 ? 3 : 2)
fwd5_kernel(const __grid_constant__ CUtensorMap xmap, const ApplyArgs<float> a, int* status,
            uint32_t slab_stride, uint32_t warp_bytes) {
    static_assert(BC >= 4 && BC <= 32, "16-byte batch records");
    constexpr int Q = BC / 4;
    constexpr int FC = 32 * FPL;
    extern __shared__ unsigned char smem6_raw[];
    const uint32_t raw_u32 = smem_u32(smem6_raw);
    const uint32_t base_u32 = (raw_u32 + 127) & ~127u;
    unsigned char* base = smem6_raw + (base_u32 - raw_u32);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // per warp: [stage 0: 4 slabs][stage 1: 4 slabs][z][2 mbarriers]
    unsigned char* wbase = base + (size_t)warp * warp_bytes;
    const uint32_t wbase_u32 = base_u32 + warp * warp_bytes;
    float4* zsv = reinterpret_cast<float4*>(wbase + 8 * slab_stride);
    const uint32_t bar0 = wbase_u32 + warp_bytes - 16;
    const uint32_t box_bytes = (uint32_t)a.zwin * BC * 4;
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int64_t warp_global = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    const int64_t n_warps = (int64_t)gridDim.x * kWarpsPerBlock;
    const uint64_t tmap = reinterpret_cast<uint64_t>(&xmap);
    struct Item {
        int64_t task;
        int e, e_end, row_out, f_begin, b0, k_lo;
    };
    auto task_item = [&](int64_t task, Item& it) {
        it.task = task;
        const int bchunk = (int)(task % a.n_bchunk);
        const int64_t t2 = task / a.n_bchunk;
        const int fchunk = (int)(t2 % a.n_fchunk);
        int row;
        task_row(a, (int)(t2 / a.n_fchunk), it.row_out, row);
        it.f_begin = fchunk * FC;
        it.b0 = bchunk * BC;
        it.e = a.row_ptr[row];
        it.e_end = a.row_ptr[row + 1];
    };
    auto set_window = [&](Item& it) {
        const int f_end = min(a.Tn, it.f_begin + FC);
        const int64_t U0 = (int64_t)a.K0[it.e] * kFracOne + (int64_t)a.F0[it.e];
        it.k_lo = (int)((U0 - (int64_t)(f_end - 1) * a.D) >> kFracBits);
    };
    auto issue = [&](const Item& it, int b) {
        if (lane != 0) return;
        const uint32_t bar = bar0 + 8u * b;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(4 * box_bytes)
                     : "memory");
        const int n00 = a.node00[it.e], n01 = a.node01[it.e];
        const int node[4] = {n00, n00 + a.n_phi, n01, n01 + a.n_phi};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t dst = wbase_u32 + (uint32_t)(4 * b + c) * slab_stride;
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
                "l"(tmap), "r"(it.b0), "r"(it.k_lo), "r"(node[c]), "r"(bar)
                : "memory");
        }
    };
    int64_t task = warp_global;
    if (task >= a.n_tasks) return;
    Item cur;
    task_item(task, cur);
    set_window(cur);
    issue(cur, 0);
    float acc[FPL][BC];
#pragma unroll
    for (int j = 0; j < FPL; ++j)
#pragma unroll
        for (int b = 0; b < BC; ++b) acc[j][b] = 0.0f;
    for (uint32_t t = 0;; ++t) {
        // the item after cur: next ray of the row, else the first ray of the next task
        Item nxt = cur;
        bool more = true;
        if (cur.e + 1 < cur.e_end) {
            ++nxt.e;
        } else if (cur.task + n_warps < a.n_tasks) {
            task_item(cur.task + n_warps, nxt);
        } else {
            more = false;
        }
        if (more) {
            set_window(nxt);
            issue(nxt, (t + 1) & 1);
        }
        if (!mbar_wait(bar0 + 8u * (t & 1), (t >> 1) & 1)) {
            if (lane == 0) atomicOr(status, 1);
            if (more) mbar_wait(bar0 + 8u * ((t + 1) & 1), ((t + 1) >> 1) & 1);
            return;
        }
        // ray cur.e: z[k][.] = sum_c W_c x[node_c][k][.] from the staged slabs
        const int f_end = min(a.Tn, cur.f_begin + FC);
        const int64_t U0 = (int64_t)a.K0[cur.e] * kFracOne + (int64_t)a.F0[cur.e];
        const int k_top = (int)((U0 - (int64_t)cur.f_begin * a.D) >> kFracBits);
        const int nwin = k_top + 2 - cur.k_lo;
        const float4 wv = corner_weights(a.W, a.W16, cur.e);
        const float4* slab = reinterpret_cast<const float4*>(wbase + (size_t)(4 * (t & 1)) * slab_stride);
        const int sv = (int)(slab_stride / 16);  // float4 per slab
        for (int o = lane; o < nwin * Q; o += 32) {
            const float4 v0 = slab[o], v1 = slab[sv + o], v2 = slab[2 * sv + o], v3 = slab[3 * sv + o];
            float4 z;
            z.x = interp4(wv.x, v0.x, wv.y, v1.x, wv.z, v2.x, wv.w, v3.x);
            z.y = interp4(wv.x, v0.y, wv.y, v1.y, wv.z, v2.y, wv.w, v3.y);
            z.z = interp4(wv.x, v0.z, wv.y, v1.z, wv.z, v2.z, wv.w, v3.z);
            z.w = interp4(wv.x, v0.w, wv.y, v1.w, wv.z, v2.w, wv.w, v3.w);
            zsv[o] = z;
        }
        __syncwarp();
        int64_t U = U0 - (int64_t)(cur.f_begin + lane) * a.D;
        const int64_t dU = (int64_t)32 * a.D;
#pragma unroll
        for (int j = 0; j < FPL; ++j) {
            const int f = cur.f_begin + lane + 32 * j;
            if (f < f_end) {
                const int k0 = (int)(U >> kFracBits);
                const float fr = (float)(int32_t)(U & kFracMask) * (1.0f / (float)kFracOne);
                const float g = 1.0f - fr;
                const float4* z0 = zsv + (k0 - cur.k_lo) * Q;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float4 p0 = z0[q], p1 = z0[Q + q];
                    acc[j][4 * q + 0] = hat2(acc[j][4 * q + 0], g, p0.x, fr, p1.x);
                    acc[j][4 * q + 1] = hat2(acc[j][4 * q + 1], g, p0.y, fr, p1.y);
                    acc[j][4 * q + 2] = hat2(acc[j][4 * q + 2], g, p0.z, fr, p1.z);
                    acc[j][4 * q + 3] = hat2(acc[j][4 * q + 3], g, p0.w, fr, p1.w);
                }
            }
            U -= dU;
        }
        __syncwarp();  // zs and stage t & 1 are free again
        if (cur.e + 1 >= cur.e_end) {  // last ray of the task: write y
            const int nb = min(BC, a.B - cur.b0);
#pragma unroll
            for (int j = 0; j < FPL; ++j) {
                const int f = cur.f_begin + lane + 32 * j;
                if (f < f_end) {
                    float* yo = a.out + ((int64_t)cur.row_out * a.Tn + f) * a.B + cur.b0;
                    if (nb == BC) {
#pragma unroll
                        for (int q = 0; q < Q; ++q)
                            reinterpret_cast<float4*>(yo)[q] = make_float4(
                                acc[j][4 * q], acc[j][4 * q + 1], acc[j][4 * q + 2], acc[j][4 * q + 3]);
                    } else {
#pragma unroll
                        for (int b = 0; b < BC; ++b)
                            if (b < nb) yo[b] = acc[j][b];
                    }
                }
#pragma unroll
                for (int b = 0; b < BC; ++b) acc[j][b] = 0.0f;
            }
        }
        if (!more) break;
        cur = nxt;
    }
}

constexpr int kFwd7Warps = 4;
constexpr int kFwd7MinBlocks = 4;

// one ray's table fields (the forward's per-ray inputs)
struct Fwd7Ray {
    int K0, F0, n00, n01;
    float4 w;
};

__device__ __forceinline__ Fwd7Ray fwd7_load_ray(const ApplyArgs<float>& a, int e) {
    Fwd7Ray r;
    if (a.ray_rec) {  // one 32-byte record: two loads from one sector
        const float4 f = a.ray_rec[2 * (int64_t)e];
        r.K0 = __float_as_int(f.x);
        r.F0 = __float_as_int(f.y);
        r.n00 = __float_as_int(f.z);
        r.n01 = __float_as_int(f.w);
        r.w = a.ray_rec[2 * (int64_t)e + 1];
    } else {
        r.K0 = a.K0[e];
        r.F0 = a.F0[e];
        r.n00 = a.node00[e];
        r.n01 = a.node01[e];
        r.w = corner_weights(a.W, a.W16, e);
    }
    return r;
}

// One ray of a periodic forward task: stage the interpolated history of the
// hats the chunk touches in shared memory, then add each lane's frames.
template <int BC, int FPL, int P>
__device__ __forceinline__ void fwd7_ray(const ApplyArgs<float>& a, const Fwd7Ray& rf, int hb, int b0,
                                         int f_begin, bool full, int lane, float4* zsv,
                                         float (&acc)[FPL][BC]) {
    constexpr int Q = BC / 4;
    constexpr int FC = 32 * FPL;
    constexpr int ZW = FC / P + 3;         // hats staged per task window
    constexpr int NU = (ZW * Q + 31) / 32;  // staging items per lane
    constexpr int HS = 32 / P;             // hat steps per 32 frames
    constexpr int32_t D = kFracOne / P;
    const int64_t KB = (int64_t)a.K * a.B;  // floats per node row of x
    const int B = a.B;                       // hat stride of x
    // this lane's staging items o = lane + 32 u: hat lane / Q + (32 / Q) u, record lane % Q
    const int kk0 = lane / Q, q0 = lane % Q;
    const int32_t lane_off = -lane * D;  // - lane D, the lane's offset inside a hat step pattern
    const int K0 = rf.K0, F0 = rf.F0;
    const float4 wv = rf.w;
    // window [k_lo, k_lo + nwin): k_top = K0 - hb, k_lo = K0 - hb - FC / P + ((F0 + D) >> 24)
    const int k_top = K0 - hb;
    const int k_lo = k_top - FC / P + ((F0 + D) >> kFracBits);
    const float* b00 = a.in + (int64_t)rf.n00 * KB + (int64_t)(k_lo + kk0) * B + b0 + 4 * q0;
    const float* b01 = a.in + (int64_t)rf.n01 * KB + (int64_t)(k_lo + kk0) * B + b0 + 4 * q0;
    const int64_t rstep = (int64_t)a.n_phi * KB;  // the radial neighbour's row
    float4 v[NU][4];
    if (k_lo >= 0 && k_lo + ZW <= a.K) {
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            if (u < NU - 1 || lane + 32 * u < ZW * Q) {
                const int du = (32 / Q) * u * B;
                v[u][0] = __ldg(reinterpret_cast<const float4*>(b00 + du));
                v[u][1] = __ldg(reinterpret_cast<const float4*>(b00 + rstep + du));
                v[u][2] = __ldg(reinterpret_cast<const float4*>(b01 + du));
                v[u][3] = __ldg(reinterpret_cast<const float4*>(b01 + rstep + du));
            }
        }
    } else {
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int k = k_lo + kk0 + (32 / Q) * u;
            const bool ok = lane + 32 * u < ZW * Q && k >= 0 && k < a.K;
            const int du = (32 / Q) * u * B;
            v[u][0] = v[u][1] = v[u][2] = v[u][3] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok) {
                v[u][0] = __ldg(reinterpret_cast<const float4*>(b00 + du));
                v[u][1] = __ldg(reinterpret_cast<const float4*>(b00 + rstep + du));
                v[u][2] = __ldg(reinterpret_cast<const float4*>(b01 + du));
                v[u][3] = __ldg(reinterpret_cast<const float4*>(b01 + rstep + du));
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        if (u < NU - 1 || lane + 32 * u < ZW * Q) {
            float2 r = __fmul2_rn(make_float2(wv.x, wv.x), make_float2(v[u][0].x, v[u][0].y));
            r = __ffma2_rn(make_float2(wv.y, wv.y), make_float2(v[u][1].x, v[u][1].y), r);
            r = __ffma2_rn(make_float2(wv.z, wv.z), make_float2(v[u][2].x, v[u][2].y), r);
            r = __ffma2_rn(make_float2(wv.w, wv.w), make_float2(v[u][3].x, v[u][3].y), r);
            float2 t = __fmul2_rn(make_float2(wv.x, wv.x), make_float2(v[u][0].z, v[u][0].w));
            t = __ffma2_rn(make_float2(wv.y, wv.y), make_float2(v[u][1].z, v[u][1].w), t);
            t = __ffma2_rn(make_float2(wv.z, wv.z), make_float2(v[u][2].z, v[u][2].w), t);
            t = __ffma2_rn(make_float2(wv.w, wv.w), make_float2(v[u][3].z, v[u][3].w), t);
            zsv[lane + 32 * u] = make_float4(r.x, r.y, t.x, t.y);
        }
    }
    __syncwarp();
    // lane's frames f_begin + lane + 32 j: remainder F0 - lane D (one value
    // per lane: 32 frames are HS whole hat steps), hat index k_top + floor
    const int32_t rem = F0 + lane_off;
    const int k00 = k_top + (rem >> kFracBits);
    const float fr = (float)(rem & kFracMask) * (1.0f / (float)kFracOne);
    const float g = 1.0f - fr;
    const float2 g2 = make_float2(g, g), f2 = make_float2(fr, fr);
    const float4* z0 = zsv + (k00 - k_lo) * Q;
#pragma unroll
    for (int j = 0; j < FPL; ++j) {
        if (full || f_begin + lane + 32 * j < a.Tn) {
#pragma unroll
            for (int qq = 0; qq < Q; ++qq) {
                const float4 p0 = z0[qq - j * HS * Q];
                const float4 p1 = z0[Q + qq - j * HS * Q];
                float2 lo = make_float2(acc[j][4 * qq], acc[j][4 * qq + 1]);
                float2 hi = make_float2(acc[j][4 * qq + 2], acc[j][4 * qq + 3]);
                lo = __ffma2_rn(g2, make_float2(p0.x, p0.y), lo);
                lo = __ffma2_rn(f2, make_float2(p1.x, p1.y), lo);
                hi = __ffma2_rn(g2, make_float2(p0.z, p0.w), hi);
                hi = __ffma2_rn(f2, make_float2(p1.z, p1.w), hi);
                acc[j][4 * qq] = lo.x;
                acc[j][4 * qq + 1] = lo.y;
                acc[j][4 * qq + 2] = hi.x;
                acc[j][4 * qq + 3] = hi.y;
            }
        }
    }
    __syncwarp();
}

// a periodic forward task's outputs: y written once, 16-byte records
template <int BC, int FPL>
__device__ __forceinline__ void fwd7_store(const ApplyArgs<float>& a, int row_out, int b0, int f_begin,
                                           bool full, int lane, const float (&acc)[FPL][BC]) {
    constexpr int Q = BC / 4;
#pragma unroll
    for (int j = 0; j < FPL; ++j) {
        const int f = f_begin + lane + 32 * j;
        if (full || f < a.Tn) {
            float4* yo = reinterpret_cast<float4*>(a.out + ((int64_t)row_out * a.Tn + f) * a.B + b0);
#pragma unroll
            for (int qq = 0; qq < Q; ++qq)
                yo[qq] = make_float4(acc[j][4 * qq], acc[j][4 * qq + 1], acc[j][4 * qq + 2],
                                     acc[j][4 * qq + 3]);
        }
    }
}

// Staged forward specialised for a periodic cadence (a frame step is 1 / P of
// a hat step, P in {2, 4, 8}) with the whole batch in one chunk (B = BC in
// {4, 8, 16}): the tasks, windows, values and accumulation order of
// fwd3_kernel<float, BC, FPL> (hence the same bits), with
//  * the hat window and each lane's hat index and fraction in exact 32-bit
//    arithmetic: a chunk starts on a whole hat step, so U(f) = U0 - f D splits
//    into K0 - f_begin / P and the 24-bit remainder F0 - (f - f_begin) D;
//  * the window size fixed at compile time (FC / P + 3 hats), so every staging
//    load, staged store and hat read is a base address plus an immediate;
//  * range tests only where a window or a chunk reaches past the hats or the
//    frames (a uniform branch per ray or task).
// 4-warp CTAs (4 per SM at <= 128 registers): the same occupancy as 8-warp
// CTAs, finer blocks for the resident grid's tail (measured faster)
template <int BC, int FPL, int P>
__global__ void __launch_bounds__(kFwd7Warps * 32, kFwd7MinBlocks)
fwd7_kernel(const ApplyArgs<float> a) {
    static_assert(BC == 4 || BC == 8 || BC == 16, "16-byte batch records");
    wait_prior_grid();
    constexpr int Q = BC / 4;
    constexpr int FC = 32 * FPL;
    static_assert(FC % P == 0, "chunks start on whole hat steps");
    constexpr int ZW = FC / P + 3;
    __shared__ __align__(16) float4 zs_all[kFwd7Warps][ZW * Q];
    float4* zsv = zs_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * kFwd7Warps + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * kFwd7Warps;
    for (TaskWalk tw(warp_global, n_warps, a.n_bchunk, a.n_fchunk); tw.r < a.seg.total; tw.next()) {
        const int b0 = tw.b * BC;
        int row_out, row;
        task_row(a, tw.r, row_out, row);
        const int f_begin = tw.f * FC;
        const bool full = f_begin + FC <= a.Tn;  // every frame of the chunk exists
        const int hb = f_begin / P;               // whole hat steps before the chunk
        float acc[FPL][BC];
#pragma unroll
        for (int j = 0; j < FPL; ++j)
#pragma unroll
            for (int b = 0; b < BC; ++b) acc[j][b] = 0.0f;
        const int e_begin = a.row_ptr[row], e_end = a.row_ptr[row + 1];
        for (int e = e_begin; e < e_end; ++e)
            fwd7_ray<BC, FPL, P>(a, fwd7_load_ray(a, e), hb, b0, f_begin, full, lane, zsv, acc);
        fwd7_store<BC, FPL>(a, row_out, b0, f_begin, full, lane, acc);
    }
}

// fwd7 with the table loads moved ahead of the work that needs them: while a
// task is processed, the next task's first ray and the row range of the task
// after it are already on their way, and inside a task the next ray's fields
// load during the current ray.  Same tasks, arithmetic and order as fwd7 (the
// same bits); 3 CTAs per SM for the extra registers.
constexpr int kFwd8MinBlocks = 3;
template <int BC, int FPL, int P>
__global__ void __launch_bounds__(kFwd7Warps * 32, kFwd8MinBlocks)
fwd8_kernel(const ApplyArgs<float> a) {
    static_assert(BC == 4 || BC == 8 || BC == 16, "16-byte batch records");
    wait_prior_grid();
    constexpr int Q = BC / 4;
    constexpr int FC = 32 * FPL;
    static_assert(FC % P == 0, "chunks start on whole hat steps");
    constexpr int ZW = FC / P + 3;
    __shared__ __align__(16) float4 zs_all[kFwd7Warps][ZW * Q];
    float4* zsv = zs_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * kFwd7Warps + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * kFwd7Warps;
    const int n_rows = a.seg.total;
    TaskWalk tw(warp_global, n_warps, a.n_bchunk, a.n_fchunk);
    if (tw.r >= n_rows) return;
    int row_out, row;
    task_row(a, tw.r, row_out, row);
    int eb = a.row_ptr[row], ee = a.row_ptr[row + 1];
    TaskWalk tn = tw;
    tn.next();
    int row_out_n = 0, eb_n = 0, ee_n = 0;
    if (tn.r < n_rows) {
        int rn;
        task_row(a, tn.r, row_out_n, rn);
        eb_n = a.row_ptr[rn];
        ee_n = a.row_ptr[rn + 1];
    }
    Fwd7Ray cur{};
    if (eb < ee) cur = fwd7_load_ray(a, eb);
    while (true) {
        // ahead: the next task's first ray, the row range of the task after it
        Fwd7Ray nxt{};
        if (tn.r < n_rows && eb_n < ee_n) nxt = fwd7_load_ray(a, eb_n);
        TaskWalk tnn = tn;
        tnn.next();
        int row_out_nn = 0, eb_nn = 0, ee_nn = 0;
        if (tnn.r < n_rows) {
            int r2;
            task_row(a, tnn.r, row_out_nn, r2);
            eb_nn = a.row_ptr[r2];
            ee_nn = a.row_ptr[r2 + 1];
        }
        const int b0 = tw.b * BC;
        const int f_begin = tw.f * FC;
        const bool full = f_begin + FC <= a.Tn;
        const int hb = f_begin / P;
        float acc[FPL][BC];
#pragma unroll
        for (int j = 0; j < FPL; ++j)
#pragma unroll
            for (int b = 0; b < BC; ++b) acc[j][b] = 0.0f;
        for (int e = eb; e < ee; ++e) {
            const Fwd7Ray rf = cur;
            if (e + 1 < ee) cur = fwd7_load_ray(a, e + 1);
            fwd7_ray<BC, FPL, P>(a, rf, hb, b0, f_begin, full, lane, zsv, acc);
        }
        fwd7_store<BC, FPL>(a, row_out, b0, f_begin, full, lane, acc);
        if (tn.r >= n_rows) break;
        tw = tn;
        row_out = row_out_n;
        eb = eb_n;
        ee = ee_n;
        cur = nxt;
        tn = tnn;
        row_out_n = row_out_nn;
        eb_n = eb_nn;
        ee_n = ee_nn;
    }
}

// Periodic forward with the batch spread over the lanes: Q = BC / 4 lanes
// share a frame, each holding one 16-byte quad of its columns, so a warp's
// store instruction writes 512 contiguous bytes of y (whole sectors and lines)
// at every batch size, where the lane-per-frame kernels (fwd7/fwd8) write
// 16-byte pieces at a BC * 4-byte stride (8 lines per instruction at BC = 8,
// 16 at BC = 16) and their stores and shared-memory reads of whole frame
// records saturate the load/store pipe as BC grows.  Lane (s, c) = (lane / Q,
// lane % Q) adds the frames f_begin + s + (32 / Q) j, j < NF, of the quad c;
// the chunk is FC = 32 NF / Q frames.  The hat window, its staging in shared
// memory (the interpolated history z of fwd7_ray, the same values), the ray
// order and each output's fused multiply-add chain are fwd7's: the same bits.
// BC in {4, 8, 16, 32, 64}; B = BC or whole chunks of BC columns.
template <int BC, int NF>
struct Fwd9Shape {
    static constexpr int Q = BC / 4;
    static constexpr int R = 32 / Q;  // frames per lane row
    static constexpr int FC = R * NF;
};

template <int BC, int NF, int P>
__device__ __forceinline__ void fwd9_ray(const ApplyArgs<float>& a, const Fwd7Ray& rf, int hb, int b0,
                                         int f_begin, bool full, int lane, float4* zsv,
                                         float4 (&acc)[NF]) {
    constexpr int Q = Fwd9Shape<BC, NF>::Q;
    constexpr int R = Fwd9Shape<BC, NF>::R;
    constexpr int FC = Fwd9Shape<BC, NF>::FC;
    constexpr int ZW = FC / P + 3;          // hats staged per task window
    constexpr int NU = (ZW * Q + 31) / 32;  // staging items per lane
    constexpr int32_t D = kFracOne / P;
    const int64_t KB = (int64_t)a.K * a.B;  // floats per node row of x
    const int B = a.B;                       // hat stride of x
    const int s = lane / Q, c = lane % Q;    // staging: hat s + (32 / Q) u, quad c
    const int K0 = rf.K0, F0 = rf.F0;
    const float4 wv = rf.w;
    const int k_top = K0 - hb;
    const int k_lo = k_top - FC / P + ((F0 + D) >> kFracBits);
    const float* b00 = a.in + (int64_t)rf.n00 * KB + (int64_t)(k_lo + s) * B + b0 + 4 * c;
    const float* b01 = a.in + (int64_t)rf.n01 * KB + (int64_t)(k_lo + s) * B + b0 + 4 * c;
    const int64_t rstep = (int64_t)a.n_phi * KB;  // the radial neighbour's row
    float4 v[NU][4];
    if (k_lo >= 0 && k_lo + ZW <= a.K) {
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            if (u < NU - 1 || lane + 32 * u < ZW * Q) {
                const int du = R * u * B;
                v[u][0] = __ldg(reinterpret_cast<const float4*>(b00 + du));
                v[u][1] = __ldg(reinterpret_cast<const float4*>(b00 + rstep + du));
                v[u][2] = __ldg(reinterpret_cast<const float4*>(b01 + du));
                v[u][3] = __ldg(reinterpret_cast<const float4*>(b01 + rstep + du));
            }
        }
    } else {
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int k = k_lo + s + R * u;
            const bool ok = lane + 32 * u < ZW * Q && k >= 0 && k < a.K;
            const int du = R * u * B;
            v[u][0] = v[u][1] = v[u][2] = v[u][3] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok) {
                v[u][0] = __ldg(reinterpret_cast<const float4*>(b00 + du));
                v[u][1] = __ldg(reinterpret_cast<const float4*>(b00 + rstep + du));
                v[u][2] = __ldg(reinterpret_cast<const float4*>(b01 + du));
                v[u][3] = __ldg(reinterpret_cast<const float4*>(b01 + rstep + du));
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        if (u < NU - 1 || lane + 32 * u < ZW * Q) {
            float2 r = __fmul2_rn(make_float2(wv.x, wv.x), make_float2(v[u][0].x, v[u][0].y));
            r = __ffma2_rn(make_float2(wv.y, wv.y), make_float2(v[u][1].x, v[u][1].y), r);
            r = __ffma2_rn(make_float2(wv.z, wv.z), make_float2(v[u][2].x, v[u][2].y), r);
            r = __ffma2_rn(make_float2(wv.w, wv.w), make_float2(v[u][3].x, v[u][3].y), r);
            float2 t = __fmul2_rn(make_float2(wv.x, wv.x), make_float2(v[u][0].z, v[u][0].w));
            t = __ffma2_rn(make_float2(wv.y, wv.y), make_float2(v[u][1].z, v[u][1].w), t);
            t = __ffma2_rn(make_float2(wv.z, wv.z), make_float2(v[u][2].z, v[u][2].w), t);
            t = __ffma2_rn(make_float2(wv.w, wv.w), make_float2(v[u][3].z, v[u][3].w), t);
            zsv[lane + 32 * u] = make_float4(r.x, r.y, t.x, t.y);
        }
    }
    __syncwarp();
    // frame f_begin + s + R j: remainder F0 - (s + R j) D (above -2^31: (FC - 1) D
    // < 128 hat steps), hat k_top + floor(remainder / 2^24), fraction its low 24 bits
    const float4* zc = zsv + c;
    const int32_t rem_s = F0 - s * D;
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        if (full || f_begin + s + R * j < a.Tn) {
            int k;
            float fr;
            if constexpr (R % P == 0) {  // every row of lanes a whole number of hat steps on
                k = k_top + (rem_s >> kFracBits) - j * (R / P);
                fr = (float)(rem_s & kFracMask) * (1.0f / (float)kFracOne);
            } else {
                const int32_t rem = rem_s - R * j * D;
                k = k_top + (rem >> kFracBits);
                fr = (float)(rem & kFracMask) * (1.0f / (float)kFracOne);
            }
            const float g = 1.0f - fr;
            const float2 g2 = make_float2(g, g), f2 = make_float2(fr, fr);
            const float4 p0 = zc[(k - k_lo) * Q];
            const float4 p1 = zc[(k + 1 - k_lo) * Q];
            float2 lo = make_float2(acc[j].x, acc[j].y);
            float2 hi = make_float2(acc[j].z, acc[j].w);
            lo = __ffma2_rn(g2, make_float2(p0.x, p0.y), lo);
            lo = __ffma2_rn(f2, make_float2(p1.x, p1.y), lo);
            hi = __ffma2_rn(g2, make_float2(p0.z, p0.w), hi);
            hi = __ffma2_rn(f2, make_float2(p1.z, p1.w), hi);
            acc[j] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
    }
    __syncwarp();
}

template <int BC, int NF>
__device__ __forceinline__ void fwd9_store(const ApplyArgs<float>& a, int row_out, int b0, int f_begin,
                                           bool full, int lane, const float4 (&acc)[NF]) {
    constexpr int Q = Fwd9Shape<BC, NF>::Q;
    constexpr int R = Fwd9Shape<BC, NF>::R;
    const int s = lane / Q, c = lane % Q;
    float* base = a.out + ((int64_t)row_out * a.Tn + f_begin + s) * a.B + b0 + 4 * c;
#pragma unroll
    for (int j = 0; j < NF; ++j)
        if (full || f_begin + s + R * j < a.Tn)
            *reinterpret_cast<float4*>(base + (int64_t)R * j * a.B) = acc[j];
}

constexpr int kFwd9Warps = 4;
// CTAs per SM the register budget is set for: four, three for 32 and more
// columns and for the prefetching form (whose next-task fields and row range
// spilled in the four-CTA budget)
template <int BC, bool PF>
struct Fwd9Occ {
    static constexpr int kMinBlocks = (BC >= 32 || PF) ? 3 : 4;
};

// PF: the table loads one task (and, inside a task, one ray) ahead, as fwd8
template <int BC, int NF, int P, bool PF>
__global__ void __launch_bounds__(kFwd9Warps * 32, Fwd9Occ<BC, PF>::kMinBlocks)
fwd9_kernel(const ApplyArgs<float> a) {
    static_assert(BC == 4 || BC == 8 || BC == 16 || BC == 32 || BC == 64, "16-byte quads");
    wait_prior_grid();
    constexpr int Q = Fwd9Shape<BC, NF>::Q;
    constexpr int FC = Fwd9Shape<BC, NF>::FC;
    static_assert(FC % P == 0, "chunks start on whole hat steps");
    static_assert(FC / P <= 128, "remainders stay above -2^31");
    constexpr int ZW = FC / P + 3;
    __shared__ __align__(16) float4 zs_all[kFwd9Warps][ZW * Q];
    float4* zsv = zs_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * kFwd9Warps + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * kFwd9Warps;
    const int n_rows = a.seg.total;
    if constexpr (!PF) {
        for (TaskWalk tw(warp_global, n_warps, a.n_bchunk, a.n_fchunk); tw.r < n_rows; tw.next()) {
            const int b0 = tw.b * BC;
            int row_out, row;
            task_row(a, tw.r, row_out, row);
            const int f_begin = tw.f * FC;
            const bool full = f_begin + FC <= a.Tn;
            const int hb = f_begin / P;
            float4 acc[NF];
#pragma unroll
            for (int j = 0; j < NF; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            const int e_begin = a.row_ptr[row], e_end = a.row_ptr[row + 1];
            for (int e = e_begin; e < e_end; ++e)
                fwd9_ray<BC, NF, P>(a, fwd7_load_ray(a, e), hb, b0, f_begin, full, lane, zsv, acc);
            fwd9_store<BC, NF>(a, row_out, b0, f_begin, full, lane, acc);
        }
    } else {
        TaskWalk tw(warp_global, n_warps, a.n_bchunk, a.n_fchunk);
        if (tw.r >= n_rows) return;
        int row_out, row;
        task_row(a, tw.r, row_out, row);
        int eb = a.row_ptr[row], ee = a.row_ptr[row + 1];
        TaskWalk tn = tw;
        tn.next();
        int row_out_n = 0, eb_n = 0, ee_n = 0;
        if (tn.r < n_rows) {
            int rn;
            task_row(a, tn.r, row_out_n, rn);
            eb_n = a.row_ptr[rn];
            ee_n = a.row_ptr[rn + 1];
        }
        Fwd7Ray cur{};
        if (eb < ee) cur = fwd7_load_ray(a, eb);
        while (true) {
            Fwd7Ray nxt{};
            if (tn.r < n_rows && eb_n < ee_n) nxt = fwd7_load_ray(a, eb_n);
            TaskWalk tnn = tn;
            tnn.next();
            int row_out_nn = 0, eb_nn = 0, ee_nn = 0;
            if (tnn.r < n_rows) {
                int r2;
                task_row(a, tnn.r, row_out_nn, r2);
                eb_nn = a.row_ptr[r2];
                ee_nn = a.row_ptr[r2 + 1];
            }
            const int b0 = tw.b * BC;
            const int f_begin = tw.f * FC;
            const bool full = f_begin + FC <= a.Tn;
            const int hb = f_begin / P;
            float4 acc[NF];
#pragma unroll
            for (int j = 0; j < NF; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int e = eb; e < ee; ++e) {
                const Fwd7Ray rf = cur;
                if (e + 1 < ee) cur = fwd7_load_ray(a, e + 1);
                fwd9_ray<BC, NF, P>(a, rf, hb, b0, f_begin, full, lane, zsv, acc);
            }
            fwd9_store<BC, NF>(a, row_out, b0, f_begin, full, lane, acc);
            if (tn.r >= n_rows) break;
            tw = tn;
            row_out = row_out_n;
            eb = eb_n;
            ee = ee_n;
            cur = nxt;
            tn = tnn;
            row_out_n = row_out_nn;
            eb_n = eb_nn;
            ee_n = ee_nn;
        }
    }
}

// Periodic forward for batches of one or two columns (forward kernels 7 and
// 8 there): each lane holds one 16-byte unit of y, the G = 4 / BC
// consecutive frames f_begin + G lane + i + 32 G j (i < G, j < NF) of all BC
// columns, so a warp's store instruction writes 512 contiguous bytes, as in
// the quad-lane kernels.  The hat window, the staged history z (one hat
// record per lane and item: a coalesced 4- or 8-byte read of each corner
// row), the ray order and each output's fused multiply-add chain are fwd7's:
// the same bits.
template <int BC, int NF>
struct Fwd11Shape {
    static constexpr int G = 4 / BC;            // frames per lane unit
    static constexpr int FC = 32 * G * NF;      // frames per task
};

template <int BC, int NF, int P>
__device__ __forceinline__ void fwd11_ray(const ApplyArgs<float>& a, const Fwd7Ray& rf, int hb,
                                          int f_begin, bool full, int lane, float* zs,
                                          float (&acc)[NF][4]) {
    constexpr int G = Fwd11Shape<BC, NF>::G;
    constexpr int FC = Fwd11Shape<BC, NF>::FC;
    constexpr int ZW = FC / P + 3;          // hats staged per task window
    constexpr int NU = (ZW + 31) / 32;      // hats per lane
    constexpr int32_t D = kFracOne / P;
    const int64_t KB = (int64_t)a.K * BC;  // floats per node row of x (B = BC)
    const int k_top = rf.K0 - hb;
    const int k_lo = k_top - FC / P + ((rf.F0 + D) >> kFracBits);
    const float* b00 = a.in + (int64_t)rf.n00 * KB;
    const float* b01 = a.in + (int64_t)rf.n01 * KB;
    const int64_t rstep = (int64_t)a.n_phi * KB;  // the radial neighbour's row
    const float4 wv = rf.w;
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        const int o = lane + 32 * u;
        const int k = k_lo + o;
        if (u < NU - 1 || o < ZW) {
            const bool ok = k >= 0 && k < a.K;
#pragma unroll
            for (int b = 0; b < BC; ++b) {
                float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
                if (ok) {
                    const int64_t off = (int64_t)k * BC + b;
                    v0 = __ldg(b00 + off);
                    v1 = __ldg(b00 + rstep + off);
                    v2 = __ldg(b01 + off);
                    v3 = __ldg(b01 + rstep + off);
                }
                float r = __fmul_rn(wv.x, v0);
                r = __fmaf_rn(wv.y, v1, r);
                r = __fmaf_rn(wv.z, v2, r);
                r = __fmaf_rn(wv.w, v3, r);
                zs[o * BC + b] = r;
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < NF; ++j) {
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int fl = G * lane + i + 32 * G * j;  // frame offset in the chunk
            if (full || f_begin + fl < a.Tn) {
                const int32_t rem = rf.F0 - fl * D;
                const int k = k_top + (rem >> kFracBits);
                const float fr = (float)(rem & kFracMask) * (1.0f / (float)kFracOne);
                const float g = 1.0f - fr;
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    const float p0 = zs[(k - k_lo) * BC + b];
                    const float p1 = zs[(k + 1 - k_lo) * BC + b];
                    float c = acc[j][i * BC + b];
                    c = __fmaf_rn(g, p0, c);
                    c = __fmaf_rn(fr, p1, c);
                    acc[j][i * BC + b] = c;
                }
            }
        }
    }
    __syncwarp();
}

template <int BC, int NF>
__device__ __forceinline__ void fwd11_store(const ApplyArgs<float>& a, int row_out, int f_begin, bool full,
                                            int lane, const float (&acc)[NF][4]) {
    constexpr int G = Fwd11Shape<BC, NF>::G;
    float* base = a.out + ((int64_t)row_out * a.Tn + f_begin + G * lane) * BC;
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        float* o = base + (int64_t)32 * G * j * BC;
        const int f0 = f_begin + G * lane + 32 * G * j;
        if (full || f0 + G <= a.Tn) {
            *reinterpret_cast<float4*>(o) = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
        } else {
#pragma unroll
            for (int i = 0; i < G; ++i)
                if (f0 + i < a.Tn)
#pragma unroll
                    for (int b = 0; b < BC; ++b) o[i * BC + b] = acc[j][i * BC + b];
        }
    }
}

// PF: the table loads one task (and, inside a task, one ray) ahead, as fwd8
template <int BC, int NF, int P, bool PF>
__global__ void __launch_bounds__(kFwd9Warps * 32, 4)
fwd11_kernel(const ApplyArgs<float> a) {
    static_assert(BC == 1 || BC == 2, "one or two columns");
    wait_prior_grid();
    constexpr int FC = Fwd11Shape<BC, NF>::FC;
    static_assert(FC % P == 0, "chunks start on whole hat steps");
    static_assert(FC / P <= 128, "remainders stay above -2^31");
    constexpr int ZW = FC / P + 3;
    __shared__ float zs_all[kFwd9Warps][ZW * BC];
    float* zs = zs_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (int64_t)blockIdx.x * kFwd9Warps + (threadIdx.x >> 5);
    const int64_t n_warps = (int64_t)gridDim.x * kFwd9Warps;
    const int n_rows = a.seg.total;
    auto zero = [&](float (&acc)[NF][4]) {
#pragma unroll
        for (int j = 0; j < NF; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][q] = 0.0f;
    };
    if constexpr (!PF) {
        for (TaskWalk tw(warp_global, n_warps, 1, a.n_fchunk); tw.r < n_rows; tw.next()) {
            int row_out, row;
            task_row(a, tw.r, row_out, row);
            const int f_begin = tw.f * FC;
            const bool full = f_begin + FC <= a.Tn;
            const int hb = f_begin / P;
            float acc[NF][4];
            zero(acc);
            const int e_begin = a.row_ptr[row], e_end = a.row_ptr[row + 1];
            for (int e = e_begin; e < e_end; ++e)
                fwd11_ray<BC, NF, P>(a, fwd7_load_ray(a, e), hb, f_begin, full, lane, zs, acc);
            fwd11_store<BC, NF>(a, row_out, f_begin, full, lane, acc);
        }
    } else {
        TaskWalk tw(warp_global, n_warps, 1, a.n_fchunk);
        if (tw.r >= n_rows) return;
        int row_out, row;
        task_row(a, tw.r, row_out, row);
        int eb = a.row_ptr[row], ee = a.row_ptr[row + 1];
        TaskWalk tn = tw;
        tn.next();
        int row_out_n = 0, eb_n = 0, ee_n = 0;
        if (tn.r < n_rows) {
            int rn;
            task_row(a, tn.r, row_out_n, rn);
            eb_n = a.row_ptr[rn];
            ee_n = a.row_ptr[rn + 1];
        }
        Fwd7Ray cur{};
        if (eb < ee) cur = fwd7_load_ray(a, eb);
        while (true) {
            Fwd7Ray nxt{};
            if (tn.r < n_rows && eb_n < ee_n) nxt = fwd7_load_ray(a, eb_n);
            TaskWalk tnn = tn;
            tnn.next();
            int row_out_nn = 0, eb_nn = 0, ee_nn = 0;
            if (tnn.r < n_rows) {
                int r2;
                task_row(a, tnn.r, row_out_nn, r2);
                eb_nn = a.row_ptr[r2];
                ee_nn = a.row_ptr[r2 + 1];
            }
            const int f_begin = tw.f * FC;
            const bool full = f_begin + FC <= a.Tn;
            const int hb = f_begin / P;
            float acc[NF][4];
            zero(acc);
            for (int e = eb; e < ee; ++e) {
                const Fwd7Ray rf = cur;
                if (e + 1 < ee) cur = fwd7_load_ray(a, e + 1);
                fwd11_ray<BC, NF, P>(a, rf, hb, f_begin, full, lane, zs, acc);
            }
            fwd11_store<BC, NF>(a, row_out, f_begin, full, lane, acc);
            if (tn.r >= n_rows) break;
            tw = tn;
            row_out = row_out_n;
            eb = eb_n;
            ee = ee_n;
            cur = nxt;
            tn = tnn;
            row_out_n = row_out_nn;
            eb_n = eb_nn;
            ee_n = ee_nn;
        }
    }
}

// Quad-lane periodic forward with the corner slabs of x staged one ray ahead
// by per-lane asynchronous copies (fwd10).  The warp walks its tasks as a
// flat sequence of slots (a ray of a task, or a task without rays): while
// slot i is contracted, the copies of slot i + 1 (16 bytes per lane and item,
// into the other of two shared-memory stages; hats outside [0, K) arrive as
// zeros) and the table fields of slot i + 2 are on their way, so no register
// holds a corner slab.  A lane combines the corner items it copied itself
// (the interpolated history z of fwd7_ray, written in place of corner 0),
// then the frames are fwd9's: the same values, order and bits.
template <int BC, int NF, int P>
struct Fwd10Shape {
    static constexpr int Q = BC / 4;
    static constexpr int R = 32 / Q;
    static constexpr int FC = R * NF;
    static constexpr int ZW = FC / P + 3;       // hats per window
    static constexpr int SW = ZW * Q;           // 16-byte items per corner slab
    static constexpr int NU = (SW + 31) / 32;   // items per lane
    static constexpr int kStage = 4 * SW;       // 16-byte items per stage
};
constexpr int kFwd10Warps = 4;

// a slot of the warp's walk: its task and (e < e_end) its ray
struct Fwd10Slot {
    int row_out, f_begin, b0, e, e_end;
    bool valid;
};

template <int BC, int NF, int P>
__global__ void __launch_bounds__(kFwd10Warps * 32, 4)
fwd10_kernel(const ApplyArgs<float> a) {
    static_assert(BC == 4 || BC == 8 || BC == 16 || BC == 32 || BC == 64, "16-byte quads");
    wait_prior_grid();
    using S = Fwd10Shape<BC, NF, P>;
    constexpr int Q = S::Q, R = S::R, FC = S::FC, SW = S::SW, NU = S::NU;
    static_assert(FC % P == 0, "chunks start on whole hat steps");
    static_assert(FC / P <= 128, "remainders stay above -2^31");
    constexpr int32_t D = kFracOne / P;
    extern __shared__ __align__(16) float4 smem_f10[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* stages = smem_f10 + (size_t)warp * 2 * S::kStage;
    const int s_l = lane / Q, c_l = lane % Q;  // the lane's hat row and column quad
    const int64_t KB = (int64_t)a.K * a.B;
    const int n_rows = a.seg.total;
    // the walk
    TaskWalk tw((int64_t)blockIdx.x * kFwd10Warps + warp, (int64_t)gridDim.x * kFwd10Warps, a.n_bchunk,
                a.n_fchunk);
    int w_row_out = 0, w_e = 0, w_ee = 0;
    bool w_valid = tw.r < n_rows;
    if (w_valid) {
        int row;
        task_row(a, tw.r, w_row_out, row);
        w_e = a.row_ptr[row];
        w_ee = a.row_ptr[row + 1];
    }
    auto take = [&](Fwd10Slot& sl) {  // the walk's current slot, then advance
        sl.valid = w_valid;
        sl.row_out = w_row_out;
        sl.f_begin = tw.f * FC;
        sl.b0 = tw.b * BC;
        sl.e = w_e;
        sl.e_end = w_ee;
        if (!w_valid) return;
        if (w_e + 1 < w_ee) {
            ++w_e;
            return;
        }
        tw.next();
        w_valid = tw.r < n_rows;
        if (w_valid) {
            int row;
            task_row(a, tw.r, w_row_out, row);
            w_e = a.row_ptr[row];
            w_ee = a.row_ptr[row + 1];
        }
    };
    // the copies of a slot's ray into stage st (its window as in fwd9_ray)
    auto issue = [&](const Fwd10Slot& sl, const Fwd7Ray& rf, int st) {
        if (sl.valid && sl.e < sl.e_end) {
            const int k_top = rf.K0 - sl.f_begin / P;
            const int k_lo = k_top - FC / P + ((rf.F0 + D) >> kFracBits);
            float4* dst0 = stages + st * S::kStage;
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                const int o = lane + 32 * u;
                if (u < NU - 1 || o < SW) {
                    const int k = k_lo + s_l + R * u;
                    const bool in = k >= 0 && k < a.K;
#pragma unroll
                    for (int cn = 0; cn < 4; ++cn) {
                        const int node = (cn < 2 ? rf.n00 : rf.n01) + (cn & 1) * a.n_phi;
                        const float* src = in ? a.in + (int64_t)node * KB + (int64_t)k * a.B + sl.b0 + 4 * c_l
                                              : a.in;
                        const uint32_t dst = smem_u32(dst0 + cn * SW + o);
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                                     "r"(in ? 16 : 0)
                                     : "memory");
                    }
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto fields = [&](const Fwd10Slot& sl) -> Fwd7Ray {
        Fwd7Ray r{};
        if (sl.valid && sl.e < sl.e_end) r = fwd7_load_ray(a, sl.e);
        return r;
    };
    Fwd10Slot s0, s1, s2;
    take(s0);
    take(s1);
    Fwd7Ray f0 = fields(s0), f1 = fields(s1);
    take(s2);
    issue(s0, f0, 0);
    float4 acc[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    int st = 0;
    while (s0.valid) {
        issue(s1, f1, st ^ 1);
        const Fwd7Ray f2 = fields(s2);  // two slots ahead
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        const bool full = s0.f_begin + FC <= a.Tn;
        if (s0.e < s0.e_end) {
            float4* stg = stages + st * S::kStage;
            const int k_top = f0.K0 - s0.f_begin / P;
            const int k_lo = k_top - FC / P + ((f0.F0 + D) >> kFracBits);
            const float4 wv = f0.w;
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                const int o = lane + 32 * u;
                if (u < NU - 1 || o < SW) {
                    const float4 v0 = stg[o], v1 = stg[SW + o], v2 = stg[2 * SW + o], v3 = stg[3 * SW + o];
                    float2 r = __fmul2_rn(make_float2(wv.x, wv.x), make_float2(v0.x, v0.y));
                    r = __ffma2_rn(make_float2(wv.y, wv.y), make_float2(v1.x, v1.y), r);
                    r = __ffma2_rn(make_float2(wv.z, wv.z), make_float2(v2.x, v2.y), r);
                    r = __ffma2_rn(make_float2(wv.w, wv.w), make_float2(v3.x, v3.y), r);
                    float2 t = __fmul2_rn(make_float2(wv.x, wv.x), make_float2(v0.z, v0.w));
                    t = __ffma2_rn(make_float2(wv.y, wv.y), make_float2(v1.z, v1.w), t);
                    t = __ffma2_rn(make_float2(wv.z, wv.z), make_float2(v2.z, v2.w), t);
                    t = __ffma2_rn(make_float2(wv.w, wv.w), make_float2(v3.z, v3.w), t);
                    stg[o] = make_float4(r.x, r.y, t.x, t.y);
                }
            }
            __syncwarp();
            const float4* zc = stg + c_l;
            const int32_t rem_s = f0.F0 - s_l * D;
#pragma unroll
            for (int j = 0; j < NF; ++j) {
                if (full || s0.f_begin + s_l + R * j < a.Tn) {
                    int k;
                    float fr;
                    if constexpr (R % P == 0) {
                        k = k_top + (rem_s >> kFracBits) - j * (R / P);
                        fr = (float)(rem_s & kFracMask) * (1.0f / (float)kFracOne);
                    } else {
                        const int32_t rem = rem_s - R * j * D;
                        k = k_top + (rem >> kFracBits);
                        fr = (float)(rem & kFracMask) * (1.0f / (float)kFracOne);
                    }
                    const float g = 1.0f - fr;
                    const float2 g2 = make_float2(g, g), f2v = make_float2(fr, fr);
                    const float4 p0 = zc[(k - k_lo) * Q];
                    const float4 p1 = zc[(k + 1 - k_lo) * Q];
                    float2 lo = make_float2(acc[j].x, acc[j].y);
                    float2 hi = make_float2(acc[j].z, acc[j].w);
                    lo = __ffma2_rn(g2, make_float2(p0.x, p0.y), lo);
                    lo = __ffma2_rn(f2v, make_float2(p1.x, p1.y), lo);
                    hi = __ffma2_rn(g2, make_float2(p0.z, p0.w), hi);
                    hi = __ffma2_rn(f2v, make_float2(p1.z, p1.w), hi);
                    acc[j] = make_float4(lo.x, lo.y, hi.x, hi.y);
                }
            }
        }
        __syncwarp();  // stage st is free for the copies issued next
        if (s0.e + 1 >= s0.e_end) {  // the task's last slot: its outputs
            fwd9_store<BC, NF>(a, s0.row_out, s0.b0, s0.f_begin, full, lane, acc);
#pragma unroll
            for (int j = 0; j < NF; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        s0 = s1;
        f0 = f1;
        s1 = s2;
        f1 = f2;
        take(s2);
        st ^= 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Forward with the corner slabs of x fetched by bulk asynchronous copies,
// pipelined over the warp's stream of (task, ray) items.  Tasks, hat windows,
// interpolation and accumulation order are those of fwd3_kernel<float, BC,
// FPL> (hence the same bits).  Per item, the in-range hats of the window are
// one contiguous run of each corner node's x row (the whole batch is one
// chunk), copied into a 3-stage ring of shared-memory slabs; hats outside
// [0, K) are not copied and interpolate to zero.  An item's task is decided
// four items ahead (row pointers), its table fields are loaded three ahead,
// its copies are issued two ahead together with a stage header holding what
// the contraction needs, so neither the table loads nor the copies wait in
// line with the arithmetic, and only the three items not yet issued occupy
// registers.  Waits are bounded as in adj_time5_kernel.
constexpr int kFwd6Warps = 4;
constexpr int kFwd6Stages = 3;
constexpr uint32_t kFwd6Header = 64;  // stage header bytes (16-byte multiple)

struct Fwd6Header {
    int row_out, f_begin, e, e_end;  // task and ray (e == e_end: a task without rays)
    int K0, F0, k_lo, ka;            // hat coordinate, window start, copied range [ka, kb)
    int kb, pad0, pad1, pad2;
    float4 w;                        // corner weights
};
static_assert(sizeof(Fwd6Header) == kFwd6Header, "stage header layout");

template <int BC, int FPL>
__global__ void __launch_bounds__(kFwd6Warps * 32, 4)
fwd6_kernel(const ApplyArgs<float> a, int* status, uint32_t slab_bytes, uint32_t stage_bytes) {
    static_assert(BC == 4 || BC == 8, "one 16-byte-aligned x row run per corner");
    constexpr int Q = BC / 4;
    constexpr int FC = 32 * FPL;
    constexpr int NS = kFwd6Stages;
    extern __shared__ __align__(16) unsigned char smem_f6[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t warp_bytes = NS * stage_bytes + 16 * ((8 * NS + 15) / 16);
    unsigned char* wbase = smem_f6 + (size_t)warp * warp_bytes;
    const uint32_t wbase_u32 = smem_u32(wbase);
    const uint32_t bar0 = wbase_u32 + (uint32_t)NS * stage_bytes;  // NS mbarriers, 8 bytes each
    if (lane == 0) {
#pragma unroll
        for (int st = 0; st < NS; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * st) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int64_t warp_global = (int64_t)blockIdx.x * kFwd6Warps + warp;
    const int64_t n_warps = (int64_t)gridDim.x * kFwd6Warps;
    struct It {
        int row_out, f_begin, e, e_end;  // task and ray
        int n00, n01, K0, F0;            // table fields of ray e
        float4 w;
    };
    TaskWalk tw(warp_global, n_warps, 1, a.n_fchunk);
    auto task_first = [&](It& it) -> bool {
        if (tw.r >= a.seg.total) return false;
        int row;
        task_row(a, tw.r, it.row_out, row);
        it.f_begin = tw.f * FC;
        it.e = a.row_ptr[row];
        it.e_end = a.row_ptr[row + 1];
        return true;
    };
    auto decide = [&](const It& prev, It& it) -> bool {
        if (prev.e + 1 < prev.e_end) {
            it.row_out = prev.row_out;
            it.f_begin = prev.f_begin;
            it.e = prev.e + 1;
            it.e_end = prev.e_end;
            return true;
        }
        tw.next();
        return task_first(it);
    };
    auto load = [&](It& it) {
        if (it.e < it.e_end) {
            it.n00 = a.node00[it.e];
            it.n01 = a.node01[it.e];
            it.K0 = a.K0[it.e];
            it.F0 = a.F0[it.e];
            it.w = corner_weights(a.W, a.W16, it.e);
        }
    };
    const int64_t KB = (int64_t)a.K * BC;  // floats per node row of x
    // copies of item it into stage st, with the stage header: lane 0 writes the
    // header and sets the expected bytes, then lane c < 4 copies corner c
    // (nodes n00, n00 + n_phi, n01, n01 + n_phi)
    auto issue = [&](const It& it, int st) {
        const int f_end = min(a.Tn, it.f_begin + FC);
        int bytes = 0, k_lo = 0, ka = 0, kb = 0;
        if (it.e < it.e_end) {
            const int64_t U0 = (int64_t)it.K0 * kFracOne + (int64_t)it.F0;
            const int k_top = (int)((U0 - (int64_t)it.f_begin * a.D) >> kFracBits);
            k_lo = (int)((U0 - (int64_t)(f_end - 1) * a.D) >> kFracBits);
            ka = max(k_lo, 0);
            kb = max(min(k_top + 2, a.K), ka);
            bytes = (kb - ka) * BC * 4;
        }
        unsigned char* stage = wbase + (size_t)st * stage_bytes;
        const uint32_t bar = bar0 + 8u * st;
        if (lane == 0) {
            Fwd6Header* h = reinterpret_cast<Fwd6Header*>(stage);
            reinterpret_cast<int4*>(h)[0] = make_int4(it.row_out, it.f_begin, it.e, it.e_end);
            reinterpret_cast<int4*>(h)[1] = make_int4(it.K0, it.F0, k_lo, ka);
            reinterpret_cast<int4*>(h)[2] = make_int4(kb, 0, 0, 0);
            h->w = it.w;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"(4 * bytes)
                         : "memory");
        }
        __syncwarp();
        if (lane < 4 && bytes > 0) {
            const int node = (lane < 2 ? it.n00 : it.n01) + (lane & 1) * a.n_phi;
            const float* src = a.in + (int64_t)node * KB + (int64_t)ka * BC;
            const uint32_t dst = smem_u32(stage) + kFwd6Header + (uint32_t)lane * slab_bytes +
                                 (uint32_t)((ka - k_lo) * BC * 4);
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
                " [%0], [%1], %2, [%3];" ::"r"(dst),
                "l"(src), "r"(bytes), "r"(bar)
                : "memory");
        }
    };
    float acc[FPL][BC];
#pragma unroll
    for (int j = 0; j < FPL; ++j)
#pragma unroll
        for (int b = 0; b < BC; ++b) acc[j][b] = 0.0f;
    // contraction of the item in stage st; false when the wait timed out
    auto compute = [&](int st, uint32_t parity) -> bool {
        if (!mbar_wait(bar0 + 8u * st, parity)) return false;
        unsigned char* stage = wbase + (size_t)st * stage_bytes;
        const Fwd6Header* hp = reinterpret_cast<const Fwd6Header*>(stage);
        const int4 h0 = reinterpret_cast<const int4*>(hp)[0];
        const int4 h1 = reinterpret_cast<const int4*>(hp)[1];
        const int kb = reinterpret_cast<const int4*>(hp)[2].x;
        const int row_out = h0.x, f_begin = h0.y, e = h0.z, e_end = h0.w;
        const int k_lo = h1.z, ka = h1.w;
        const int f_end = min(a.Tn, f_begin + FC);
        if (e < e_end) {
            // z[k][.] = sum_c W_c x[node_c][k][.] in place of slab 0 (zero outside [ka, kb))
            float4* s0 = reinterpret_cast<float4*>(stage + kFwd6Header);
            const int sv = (int)(slab_bytes / 16);
            const int64_t U0 = (int64_t)h1.x * kFracOne + (int64_t)h1.y;
            const int k_top = (int)((U0 - (int64_t)f_begin * a.D) >> kFracBits);
            const int nwin = k_top + 2 - k_lo;
            const int oa = (ka - k_lo) * Q, ob = (kb - k_lo) * Q;
            const float4 wv = hp->w;
            for (int base = 0; base < nwin * Q; base += 96) {
                float4 zz[3];
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    const int o = base + lane + 32 * u;
                    zz[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (o >= oa && o < ob) {
                        const float4 v0 = s0[o], v1 = s0[sv + o], v2 = s0[2 * sv + o], v3 = s0[3 * sv + o];
                        float2 r = __fmul2_rn(make_float2(wv.x, wv.x), make_float2(v0.x, v0.y));
                        r = __ffma2_rn(make_float2(wv.y, wv.y), make_float2(v1.x, v1.y), r);
                        r = __ffma2_rn(make_float2(wv.z, wv.z), make_float2(v2.x, v2.y), r);
                        r = __ffma2_rn(make_float2(wv.w, wv.w), make_float2(v3.x, v3.y), r);
                        float2 q = __fmul2_rn(make_float2(wv.x, wv.x), make_float2(v0.z, v0.w));
                        q = __ffma2_rn(make_float2(wv.y, wv.y), make_float2(v1.z, v1.w), q);
                        q = __ffma2_rn(make_float2(wv.z, wv.z), make_float2(v2.z, v2.w), q);
                        q = __ffma2_rn(make_float2(wv.w, wv.w), make_float2(v3.z, v3.w), q);
                        zz[u] = make_float4(r.x, r.y, q.x, q.y);
                    }
                }
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    const int o = base + lane + 32 * u;
                    if (o < nwin * Q) s0[o] = zz[u];
                }
            }
            __syncwarp();
            const float* zs = reinterpret_cast<const float*>(s0);
            auto add_frame = [&](int j, int k0, float fr) {
                const float g = 1.0f - fr;
                const float* z0 = zs + (k0 - k_lo) * BC;
                const float2 g2 = make_float2(g, g), f2 = make_float2(fr, fr);
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float4 p0 = reinterpret_cast<const float4*>(z0)[q];
                    const float4 p1 = reinterpret_cast<const float4*>(z0 + BC)[q];
                    float2 lo = make_float2(acc[j][4 * q], acc[j][4 * q + 1]);
                    float2 hi = make_float2(acc[j][4 * q + 2], acc[j][4 * q + 3]);
                    lo = __ffma2_rn(g2, make_float2(p0.x, p0.y), lo);
                    lo = __ffma2_rn(f2, make_float2(p1.x, p1.y), lo);
                    hi = __ffma2_rn(g2, make_float2(p0.z, p0.w), hi);
                    hi = __ffma2_rn(f2, make_float2(p1.z, p1.w), hi);
                    acc[j][4 * q] = lo.x;
                    acc[j][4 * q + 1] = lo.y;
                    acc[j][4 * q + 2] = hi.x;
                    acc[j][4 * q + 3] = hi.y;
                }
            };
            const int64_t U1 = U0 - (int64_t)(f_begin + lane) * a.D;
            if (a.hs32 > 0) {
                const int k00 = (int)(U1 >> kFracBits);
                const float fr0 = (float)(int32_t)(U1 & kFracMask) * (1.0f / (float)kFracOne);
#pragma unroll
                for (int j = 0; j < FPL; ++j)
                    if (f_begin + lane + 32 * j < f_end) add_frame(j, k00 - j * a.hs32, fr0);
            } else {
                int64_t U = U1;
                const int64_t dU = (int64_t)32 * a.D;
#pragma unroll
                for (int j = 0; j < FPL; ++j) {
                    if (f_begin + lane + 32 * j < f_end)
                        add_frame(j, (int)(U >> kFracBits),
                                  (float)(int32_t)(U & kFracMask) * (1.0f / (float)kFracOne));
                    U -= dU;
                }
            }
        }
        // z and the header were read or written by the generic proxy: order
        // those accesses before the asynchronous copies that refill the stage
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();  // the stage is free for the copies issued at the next step
        if (e + 1 >= e_end) {  // last ray of the task: write y
#pragma unroll
            for (int j = 0; j < FPL; ++j) {
                const int f = f_begin + lane + 32 * j;
                if (f < f_end) {
                    float4* yo = reinterpret_cast<float4*>(a.out + ((int64_t)row_out * a.Tn + f) * BC);
#pragma unroll
                    for (int q = 0; q < Q; ++q)
                        yo[q] = make_float4(acc[j][4 * q], acc[j][4 * q + 1], acc[j][4 * q + 2],
                                            acc[j][4 * q + 3]);
                }
#pragma unroll
                for (int b = 0; b < BC; ++b) acc[j][b] = 0.0f;
            }
        }
        return true;
    };
    // prologue: items 0 and 1 issued to stages 0 and 1, item 2 loaded, item 3 decided
    It r_[3];
    bool h_[3];
    bool have0, have1;
    {
        It i0, i1;
        have0 = task_first(i0);
        if (!have0) return;
        load(i0);
        have1 = decide(i0, i1);
        if (have1) load(i1);
        issue(i0, 0);
        if (have1) issue(i1, 1);
        h_[0] = have1 && decide(i1, r_[0]);  // item 2 (issued at step 0)
        if (h_[0]) load(r_[0]);
        h_[1] = h_[0] && decide(r_[0], r_[1]);  // item 3
    }
    // item t computes from stage t % 3; at step t the register slots hold items
    // t + 2 (issued now into stage (t + 2) % 3), t + 3 (loaded now), t + 4
    // (decided now); have_c / have_d: items t + 1 and t are in flight
    bool have_d = have0, have_c = have1;
    uint32_t ph = 0;
    auto step = [&](const int st, It& B, bool& hB, It& A, bool& hA, It& N, bool& hN) -> bool {
        if (!have_d) return false;
        const int st2 = (st + 2) % NS;
        if (hB) issue(B, st2);
        if (hA) load(A);
        hN = hA && decide(A, N);
        if (!compute(st, ph)) {
            if (lane == 0) atomicOr(status, 1);
            const int st1 = (st + 1) % NS;
            if (have_c) mbar_wait(bar0 + 8u * st1, st1 > st ? ph : ph ^ 1u);
            if (hB) mbar_wait(bar0 + 8u * st2, st2 > st ? ph : ph ^ 1u);
            return false;
        }
        have_d = have_c;
        have_c = hB;
        if (st == NS - 1) ph ^= 1u;
        return true;
    };
    for (;;) {
        if (!step(0, r_[0], h_[0], r_[1], h_[1], r_[2], h_[2])) break;
        if (!step(1, r_[1], h_[1], r_[2], h_[2], r_[0], h_[0])) break;
        if (!step(2, r_[2], h_[2], r_[0], h_[0], r_[1], h_[1])) break;
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

// 16-byte vector access is used only when the batch stride and both buffers
// allow it
template <typename T>
static int vec_ok(const ApplyArgs<T>& a) {
    constexpr int W = Vec16<T>::W;
    return (a.B % W == 0) && ((uintptr_t)a.in % 16 == 0) && ((uintptr_t)a.out % 16 == 0) ? 1 : 0;
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
    a.W16 = op->W16;
    a.W64 = op->W64;
    a.K0 = op->K0;
    a.ray_rec = op->ray_rec;
    a.F0 = op->F0;
    a.F64 = op->F64;
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
    a.status = op->dev_status;
    a.hs32 = (op->frame_D > 0 && ((int64_t)32 * op->frame_D) % kFracOne == 0)
                 ? (int)((int64_t)32 * op->frame_D / kFracOne)
                 : 0;
    return a;
}

template <typename T, int BC, int FPL, int SU = 2>
static cudaError_t launch_fwd3_bc(ApplyArgs<T> a, cudaStream_t st) {
    a.FC = 32 * FPL;
    a.vec4 = vec_ok(a);
    a.zwin = (int)ceil((a.FC - 1) * a.delta) + 3;
    a.n_fchunk = (a.Tn + a.FC - 1) / a.FC;
    a.n_bchunk = (a.B + BC - 1) / BC;
    a.n_tasks = (int64_t)a.seg.total * a.n_fchunk * a.n_bchunk;
    if (a.n_tasks == 0) return cudaSuccess;
    const size_t smem = (size_t)kWarpsPerBlock * a.zwin * BC * sizeof(T);
    if (smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(fwd3_kernel<T, BC, FPL, SU>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    const int grid =
        resident_grid(fwd3_kernel<T, BC, FPL, SU>, kWarpsPerBlock * 32, smem, a.n_tasks, kWarpsPerBlock);
    fwd3_kernel<T, BC, FPL, SU><<<grid, kWarpsPerBlock * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int BC, int P>
static cudaError_t launch_fwd4(ApplyArgs<float> a, cudaStream_t st) {
    a.vec4 = vec_ok(a);
    a.n_fchunk = (a.Tn + 32 * P - 1) / (32 * P);
    a.n_bchunk = (a.B + BC - 1) / BC;
    a.n_tasks = (int64_t)a.seg.total * a.n_fchunk * a.n_bchunk;
    if (a.n_tasks == 0) return cudaSuccess;
    fwd4_kernel<BC, P><<<grid_for(a.n_tasks), kWarpsPerBlock * 32, 0, st>>>(a);
    return cudaGetLastError();
}

// TMA forward; cudaErrorNotSupported when the batch layout cannot use it
template <int BC, int FPL>
static cudaError_t launch_fwd5(ApplyArgs<float> a, cudaStream_t st) {
    if constexpr (BC < 4) {
        return cudaErrorNotSupported;
    } else {
        if (!vec_ok(a) || !a.status) return cudaErrorNotSupported;
        const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (!enc) return cudaErrorNotSupported;
        a.FC = 32 * FPL;
        a.zwin = (int)ceil((a.FC - 1) * a.delta) + 3;
        if (a.zwin > 256) return cudaErrorNotSupported;  // TMA box rows
        a.n_fchunk = (a.Tn + a.FC - 1) / a.FC;
        a.n_bchunk = (a.B + BC - 1) / BC;
        a.n_tasks = (int64_t)a.seg.total * a.n_fchunk * a.n_bchunk;
        if (a.n_tasks == 0) return cudaSuccess;
        CUtensorMap m;
        // x as a 3D tensor: batch (inner) x hats x nodes
        cuuint64_t dims[3] = {(cuuint64_t)a.B, (cuuint64_t)a.K, (cuuint64_t)a.n_nodes};
        cuuint64_t strides[2] = {(cuuint64_t)a.B * 4, (cuuint64_t)a.K * a.B * 4};
        cuuint32_t box[3] = {(cuuint32_t)BC, (cuuint32_t)a.zwin, 1};
        cuuint32_t es[3] = {1, 1, 1};
        if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(a.in), dims, strides, box,
                es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
        // per warp: 2 stages x 4 corner slabs (128-byte aligned), z, 2 mbarriers
        const uint32_t slab_stride = ((uint32_t)a.zwin * BC * 4 + 127) & ~127u;
        const uint32_t z_bytes = ((uint32_t)a.zwin * BC * 4 + 127) & ~127u;
        const uint32_t warp_bytes = 8 * slab_stride + z_bytes + 128;  // last 16 bytes: mbarriers
        const size_t smem = 128 + (size_t)kWarpsPerBlock * warp_bytes;
        if (smem > 227 * 1024) return cudaErrorNotSupported;
        cudaError_t e = cudaFuncSetAttribute(fwd5_kernel<BC, FPL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fwd5_kernel<BC, FPL><<<grid_for(a.n_tasks), kWarpsPerBlock * 32, smem, st>>>(
            m, a, a.status, slab_stride, warp_bytes);
        return cudaGetLastError();
    }
}

// pipelined bulk-copy forward; cudaErrorNotSupported unless the whole batch
// (B = BC in {4, 8}) is one chunk of 16-byte-aligned records
template <int BC, int FPL>
static cudaError_t launch_fwd6(ApplyArgs<float> a, cudaStream_t st) {
    if (!vec_ok(a) || a.B != BC || !a.status) return cudaErrorNotSupported;
    a.FC = 32 * FPL;
    a.zwin = (int)ceil((a.FC - 1) * a.delta) + 3;
    a.n_fchunk = (a.Tn + a.FC - 1) / a.FC;
    a.n_bchunk = 1;
    a.n_tasks = (int64_t)a.seg.total * a.n_fchunk;
    if (a.n_tasks == 0) return cudaSuccess;
    // per warp: 3 stages (64-byte header, 4 corner slabs of zwin hats), then 3 mbarriers
    const uint32_t slab = ((uint32_t)a.zwin * BC * 4 + 15) & ~15u;
    const uint32_t stage = kFwd6Header + 4 * slab;
    const uint32_t warp_bytes = (uint32_t)kFwd6Stages * stage + 16 * ((8 * kFwd6Stages + 15) / 16);
    const size_t smem = (size_t)kFwd6Warps * warp_bytes;
    if (smem > 227 * 1024) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(fwd6_kernel<BC, FPL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = resident_grid(fwd6_kernel<BC, FPL>, kFwd6Warps * 32, smem, a.n_tasks, kFwd6Warps);
    fwd6_kernel<BC, FPL><<<grid, kFwd6Warps * 32, smem, st>>>(a, a.status, slab, stage);
    return cudaGetLastError();
}

// periodic one-chunk staged forward; cudaErrorNotSupported unless the
// cadence is P in {2, 4, 8} frames per hat and the whole batch (B = BC in
// {4, 8}) is one chunk of 16-byte-aligned records
template <int BC, int FPL>
static cudaError_t launch_fwd7(ApplyArgs<float> a, cudaStream_t st, bool prefetch) {
    const int P = frames_per_hat(a.D);
    if (!vec_ok(a) || a.B % BC != 0 || P == 0 || (32 * FPL) % P != 0) return cudaErrorNotSupported;
    a.FC = 32 * FPL;
    a.n_fchunk = (a.Tn + a.FC - 1) / a.FC;
    a.n_bchunk = (a.Bcols > 0 ? a.Bcols : a.B) / BC;
    a.n_tasks = (int64_t)a.seg.total * a.n_fchunk * a.n_bchunk;
    if (a.n_tasks == 0) return cudaSuccess;
    auto go = [&](auto kern) {
        const int grid = resident_grid(kern, kFwd7Warps * 32, 0, a.n_tasks, kFwd7Warps);
        return launch_dependent(kern, dim3(grid), dim3(kFwd7Warps * 32), 0, st, a);
    };
    if (prefetch) {
        switch (P) {
            case 2: return go(fwd8_kernel<BC, FPL, 2>);
            case 4: return go(fwd8_kernel<BC, FPL, 4>);
            default: return go(fwd8_kernel<BC, FPL, 8>);
        }
    }
    switch (P) {
        case 2: return go(fwd7_kernel<BC, FPL, 2>);
        case 4: return go(fwd7_kernel<BC, FPL, 4>);
        default: return go(fwd7_kernel<BC, FPL, 8>);
    }
}

// periodic quad-lane forward (fwd9); cudaErrorNotSupported unless the cadence
// is P in {2, 4, 8} frames per hat and the batch is whole chunks of BC columns
template <int BC, int NF>
static cudaError_t launch_fwd9(ApplyArgs<float> a, cudaStream_t st, bool prefetch) {
    const int P = frames_per_hat(a.D);
    constexpr int FC = Fwd9Shape<BC, NF>::FC;
    const int cols = a.Bcols > 0 ? a.Bcols : a.B;
    if (!vec_ok(a) || cols % BC != 0 || P == 0 || FC % P != 0) return cudaErrorNotSupported;
    a.FC = FC;
    a.n_fchunk = (a.Tn + FC - 1) / FC;
    a.n_bchunk = cols / BC;
    a.n_tasks = (int64_t)a.seg.total * a.n_fchunk * a.n_bchunk;
    if (a.n_tasks == 0) return cudaSuccess;
    auto go = [&](auto kern) {
        const int grid = resident_grid(kern, kFwd9Warps * 32, 0, a.n_tasks, kFwd9Warps);
        return launch_dependent(kern, dim3(grid), dim3(kFwd9Warps * 32), 0, st, a);
    };
    if (prefetch) {
        switch (P) {
            case 2: return go(fwd9_kernel<BC, NF, 2, true>);
            case 4: return go(fwd9_kernel<BC, NF, 4, true>);
            default: return go(fwd9_kernel<BC, NF, 8, true>);
        }
    }
    switch (P) {
        case 2: return go(fwd9_kernel<BC, NF, 2, false>);
        case 4: return go(fwd9_kernel<BC, NF, 4, false>);
        default: return go(fwd9_kernel<BC, NF, 8, false>);
    }
}

// the forward of a 1- or 2-column batch (fwd11); cudaErrorNotSupported
// unless the cadence is periodic, B = BC and a data row's frames are whole
// 16-byte units (T BC a multiple of 4)
template <int BC, int NF>
static cudaError_t launch_fwd11(ApplyArgs<float> a, cudaStream_t st, bool prefetch) {
    const int P = frames_per_hat(a.D);
    constexpr int FC = Fwd11Shape<BC, NF>::FC;
    if (a.B != BC || a.Bcols > 0 || P == 0 || FC % P != 0 || ((int64_t)a.Tn * BC) % 4 != 0 ||
        ((uintptr_t)a.out % 16) != 0)
        return cudaErrorNotSupported;
    a.FC = FC;
    a.n_fchunk = (a.Tn + FC - 1) / FC;
    a.n_bchunk = 1;
    a.n_tasks = (int64_t)a.seg.total * a.n_fchunk;
    if (a.n_tasks == 0) return cudaSuccess;
    auto go = [&](auto kern) {
        const int grid = resident_grid(kern, kFwd9Warps * 32, 0, a.n_tasks, kFwd9Warps);
        return launch_dependent(kern, dim3(grid), dim3(kFwd9Warps * 32), 0, st, a);
    };
    if (prefetch) {
        switch (P) {
            case 2: return go(fwd11_kernel<BC, NF, 2, true>);
            case 4: return go(fwd11_kernel<BC, NF, 4, true>);
            default: return go(fwd11_kernel<BC, NF, 8, true>);
        }
    }
    switch (P) {
        case 2: return go(fwd11_kernel<BC, NF, 2, false>);
        case 4: return go(fwd11_kernel<BC, NF, 4, false>);
        default: return go(fwd11_kernel<BC, NF, 8, false>);
    }
}

// quad-lane forward with asynchronous corner staging (fwd10); the same
// conditions as launch_fwd9
template <int BC, int NF>
static cudaError_t launch_fwd10(ApplyArgs<float> a, cudaStream_t st) {
    const int P = frames_per_hat(a.D);
    constexpr int FC = Fwd9Shape<BC, NF>::FC;
    const int cols = a.Bcols > 0 ? a.Bcols : a.B;
    if (!vec_ok(a) || cols % BC != 0 || P == 0 || FC % P != 0) return cudaErrorNotSupported;
    a.FC = FC;
    a.n_fchunk = (a.Tn + FC - 1) / FC;
    a.n_bchunk = cols / BC;
    a.n_tasks = (int64_t)a.seg.total * a.n_fchunk * a.n_bchunk;
    if (a.n_tasks == 0) return cudaSuccess;
    auto go = [&](auto kern, int stage_items) -> cudaError_t {
        const size_t smem = (size_t)kFwd10Warps * 2 * stage_items * 16;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int grid = resident_grid(kern, kFwd10Warps * 32, smem, a.n_tasks, kFwd10Warps);
        return launch_dependent(kern, dim3(grid), dim3(kFwd10Warps * 32), smem, st, a);
    };
    switch (P) {
        case 2: return go(fwd10_kernel<BC, NF, 2>, Fwd10Shape<BC, NF, 2>::kStage);
        case 4: return go(fwd10_kernel<BC, NF, 4>, Fwd10Shape<BC, NF, 4>::kStage);
        default: return go(fwd10_kernel<BC, NF, 8>, Fwd10Shape<BC, NF, 8>::kStage);
    }
}

// the default quad-lane chunk for a batch: the largest of 32, 16, 8, 4 that
// divides it (0 when the batch is not whole 16-byte records); 64-column chunks
// (16-frame tasks) measured slower than 32 (stress1024, batch 64: 33.6 vs
// 25.9 ms) and are left to the tuner
static int quad_bc(int B) {
    for (int bc = 32; bc >= 4; bc >>= 1)
        if (B % bc == 0) return bc;
    return 0;
}

int adjoint_best_kind(const rtt_op_s* op, int batch);

ApplyVariant variant_for(const rtt_op_s* op, int batch) {
    for (int i = 0; i < op->n_tuned; ++i)
        if (op->tuned_batch[i] == batch) return op->tuned[i];
    // default rule, from the kerr256 measurements: the periodic one-chunk
    // forward and the widest TMA adjoint items; each falls back to the next
    // kernel down where the cadence, batch or buffers do not allow it
    ApplyVariant v;
    const int P = frames_per_hat(op->frame_D);
    // the periodic quad-lane forward takes any batch of whole 16-byte records,
    // in chunks of up to 32 columns
    if (P > 0 && batch % 4 == 0) {
        v.fwd = 7;
        v.fwd_bc = (int8_t)quad_bc(batch);
    } else if (P > 0 && batch <= 2) {  // 16-byte units of G = 4 / B frames
        v.fwd = 7;
        v.fwd_bc = (int8_t)batch;
    } else {
        v.fwd = 1;
        v.fwd_bc = (int8_t)pick_bc(batch);
    }
    v.adj = (int8_t)adjoint_best_kind(op, batch);
    return v;
}

// staged forward with BC batch entries and (half = false) 32 / BC frames per
// lane, or (half = true, FP32 only) half as many
template <typename T, int BC>
static cudaError_t launch_fwd3_fpl(const ApplyArgs<T>& a, bool half, int su, cudaStream_t st) {
    constexpr int F = BC >= 32 ? 1 : 32 / BC;
    if constexpr (sizeof(T) == 4 && F >= 2) {
        if (half) return launch_fwd3_bc<T, BC, F / 2>(a, st);
    }
    if constexpr (sizeof(T) == 4 && (BC == 4 || BC == 8)) {
        if (su == 1) return launch_fwd3_bc<T, BC, F, 1>(a, st);
        if (su == 3) return launch_fwd3_bc<T, BC, F, 3>(a, st);
    }
    return launch_fwd3_bc<T, BC, F>(a, st);
}

template <typename T>
static cudaError_t launch_fwd3_any(const ApplyArgs<T>& a, int bc, bool half, int su,
                                   cudaStream_t st) {
    switch (bc) {
        case 1: return launch_fwd3_fpl<T, 1>(a, half, su, st);
        case 2: return launch_fwd3_fpl<T, 2>(a, half, su, st);
        case 4: return launch_fwd3_fpl<T, 4>(a, half, su, st);
        case 8: return launch_fwd3_fpl<T, 8>(a, half, su, st);
        case 16: return launch_fwd3_fpl<T, 16>(a, half, su, st);
        default: return launch_fwd3_fpl<T, 32>(a, half, su, st);
    }
}

template <int P>
static cudaError_t launch_fwd4_any(const ApplyArgs<float>& a, int bc, cudaStream_t st) {
    constexpr int BCmax = 32 / P < 8 ? 32 / P : 8;
    if (bc <= 1) return launch_fwd4<1, P>(a, st);
    if (bc <= 2) return launch_fwd4<2, P>(a, st);
    if (bc <= 4 || BCmax <= 4) return launch_fwd4<(BCmax < 4 ? BCmax : 4), P>(a, st);
    return launch_fwd4<BCmax, P>(a, st);
}

template <typename T>
cudaError_t launch_forward(const rtt_op_s* op, const T* x, T* y, int B, const ArmSeg& seg,
                           cudaStream_t st) {
    ApplyArgs<T> a = base_args<T>(op, x, y, B, seg);
    if constexpr (sizeof(T) == 4) {
        const ApplyVariant v = variant_for(op, B);
        a.row_sched = v.fwd_order ? op->row_sched : nullptr;
        const int bc = v.fwd_bc > 0 ? v.fwd_bc : pick_bc(B);
        if (v.fwd == 2) {
            switch (frames_per_hat(a.D)) {
                case 2: return launch_fwd4_any<2>(a, bc, st);
                case 4: return launch_fwd4_any<4>(a, bc, st);
                case 8: return launch_fwd4_any<8>(a, bc, st);
                default: break;  // not a periodic cadence: staged kernel
            }
        }
        if (v.fwd == 9 && (bc == 4 || bc == 8 || bc == 16 || bc == 32 || bc == 64)) {
            const bool half = v.fwd_half != 0;
            cudaError_t e;
            switch (bc) {
                case 4: e = half ? launch_fwd10<4, 4>(a, st) : launch_fwd10<4, 8>(a, st); break;
                case 8: e = half ? launch_fwd10<8, 4>(a, st) : launch_fwd10<8, 8>(a, st); break;
                case 16: e = half ? launch_fwd10<16, 4>(a, st) : launch_fwd10<16, 8>(a, st); break;
                case 32: e = half ? launch_fwd10<32, 4>(a, st) : launch_fwd10<32, 8>(a, st); break;
                default: e = half ? launch_fwd10<64, 4>(a, st) : launch_fwd10<64, 8>(a, st); break;
            }
            if (e != cudaErrorNotSupported) return e;
            cudaGetLastError();  // clear the "not supported" marker, if any
        }
        if ((v.fwd == 7 || v.fwd == 8) && (bc == 1 || bc == 2) && B == bc) {
            // frames of one or two columns in 16-byte units: NF = 2 (BC = 1) or 4
            // (BC = 2) units per lane, 256 frames per task (half: 128)
            const bool half = v.fwd_half != 0, pf = v.fwd == 8;
            const cudaError_t e = bc == 1 ? (half ? launch_fwd11<1, 1>(a, st, pf) : launch_fwd11<1, 2>(a, st, pf))
                                          : (half ? launch_fwd11<2, 2>(a, st, pf) : launch_fwd11<2, 4>(a, st, pf));
            if (e != cudaErrorNotSupported) return e;
            cudaGetLastError();  // clear the "not supported" marker, if any
        }
        if ((v.fwd == 7 || v.fwd == 8) && (bc == 4 || bc == 8 || bc == 16 || bc == 32 || bc == 64)) {
            const bool half = v.fwd_half != 0, pf = v.fwd == 8;
            // NF = 8 frames per lane (half: 4), FC = 32 NF / (BC / 4) frames per task
            cudaError_t e;
            switch (bc) {
                case 4: e = half ? launch_fwd9<4, 4>(a, st, pf) : launch_fwd9<4, 8>(a, st, pf); break;
                case 8: e = half ? launch_fwd9<8, 4>(a, st, pf) : launch_fwd9<8, 8>(a, st, pf); break;
                case 16: e = half ? launch_fwd9<16, 4>(a, st, pf) : launch_fwd9<16, 8>(a, st, pf); break;
                case 32: e = half ? launch_fwd9<32, 4>(a, st, pf) : launch_fwd9<32, 8>(a, st, pf); break;
                default: e = half ? launch_fwd9<64, 4>(a, st, pf) : launch_fwd9<64, 8>(a, st, pf); break;
            }
            if (e != cudaErrorNotSupported) return e;
            cudaGetLastError();  // clear the "not supported" marker, if any
        }
        if ((v.fwd == 5 || v.fwd == 6) && (bc == 4 || bc == 8 || bc == 16)) {
            const bool half = v.fwd_half != 0, pf = v.fwd == 6;
            auto go = [&](const ApplyArgs<float>& aa) {
                if (bc == 16) return half ? launch_fwd7<16, 1>(aa, st, pf) : launch_fwd7<16, 2>(aa, st, pf);
                return bc == 4 ? (half ? launch_fwd7<4, 4>(aa, st, pf) : launch_fwd7<4, 8>(aa, st, pf))
                               : (half ? launch_fwd7<8, 2>(aa, st, pf) : launch_fwd7<8, 4>(aa, st, pf));
            };
            cudaError_t e;
            const int pc = v.fwd_cols;
            if (pc > 0 && pc < B && B % pc == 0 && pc % bc == 0) {
                // column passes: the whole operator for pc columns at a time
                // (x's and y's working set per pass is that of a pc-column batch)
                e = cudaSuccess;
                for (int b0 = 0; b0 < B && e == cudaSuccess; b0 += pc) {
                    ApplyArgs<float> ap = a;
                    ap.in = x + b0;
                    ap.out = y + b0;
                    ap.Bcols = pc;
                    e = go(ap);
                }
            } else {
                e = go(a);
            }
            if (e != cudaErrorNotSupported) return e;
            cudaGetLastError();  // clear the "not supported" marker, if any
        }
        if (v.fwd == 4 && (bc == 4 || bc == 8)) {
            const bool half = v.fwd_half != 0;
            const cudaError_t e = bc == 4 ? (half ? launch_fwd6<4, 4>(a, st) : launch_fwd6<4, 8>(a, st))
                                          : (half ? launch_fwd6<8, 2>(a, st) : launch_fwd6<8, 4>(a, st));
            if (e != cudaErrorNotSupported) return e;
            cudaGetLastError();  // clear the "not supported" marker, if any
        }
        if (v.fwd == 3 && bc >= 4) {
            const bool half = v.fwd_half != 0;
            cudaError_t e = cudaErrorNotSupported;
            switch (bc) {
                case 4: e = half ? launch_fwd5<4, 4>(a, st) : launch_fwd5<4, 8>(a, st); break;
                case 8: e = half ? launch_fwd5<8, 2>(a, st) : launch_fwd5<8, 4>(a, st); break;
                case 16: e = half ? launch_fwd5<16, 1>(a, st) : launch_fwd5<16, 2>(a, st); break;
                default: e = launch_fwd5<32, 1>(a, st); break;
            }
            if (e != cudaErrorNotSupported) return e;
            cudaGetLastError();  // clear the "not supported" marker, if any
        }
        return launch_fwd3_any<T>(a, bc, v.fwd_half != 0, v.fwd_su, st);
    } else {
        return launch_fwd3_any<T>(a, pick_bc(B), false, 2, st);
    }
}

template cudaError_t launch_forward<float>(const rtt_op_s*, const float*, float*, int, const ArmSeg&,
                                           cudaStream_t);
template cudaError_t launch_forward<double>(const rtt_op_s*, const double*, double*, int,
                                            const ArmSeg&, cudaStream_t);

}  // namespace rtt
