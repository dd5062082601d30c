// Order mixing of whitened data (Sec. 3.1 Eq. 4):
//   d_L = C_L^{-1/2} (L (x) I) d_R,   C_L = (L (x) I) C_R (L^T (x) I),
// with C_R = I (the rows of A are already whitened), so the collapsed noise is
// the propagated one and no arm gets a noise level of its own (Sec. 4.2).
//   unresolved image: L sums, per pixel, the arm's rows of that pixel over the
//     orders; C_L = diag(c_p), c_p the pixel's row count; output rows are the
//     pixels in ascending order.
//   total flux: L sums every row of the arm; C_L = R (one output row).
// The adjoint is W^T: every row receives its output row scaled by the same
// 1 / sqrt(count).  Sums run in a fixed order (orders ascending within a
// pixel; for the total flux, fixed row blocks summed in order, then the
// blocks' sums by a fixed lane split and shuffle tree), so results are
// bitwise repeatable.  HBM bound: the mixed data is read or
// written once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "rtt_internal.cuh"

namespace rtt {

template <typename T> struct MixVec;
template <> struct MixVec<float> { using V = float4; static constexpr int W = 4; };
template <> struct MixVec<double> { using V = double2; static constexpr int W = 2; };

__device__ __forceinline__ void vadd(float4& a, const float4& b) {
    a.x = a.x + b.x; a.y = a.y + b.y; a.z = a.z + b.z; a.w = a.w + b.w;
}
__device__ __forceinline__ void vadd(double2& a, const double2& b) {
    a.x = a.x + b.x; a.y = a.y + b.y;
}
__device__ __forceinline__ void vadd(float& a, const float& b) { a = a + b; }
__device__ __forceinline__ void vadd(double& a, const double& b) { a = a + b; }
__device__ __forceinline__ void vscale(float4& a, float s) { a.x *= s; a.y *= s; a.z *= s; a.w *= s; }
__device__ __forceinline__ void vscale(double2& a, double s) { a.x *= s; a.y *= s; }
__device__ __forceinline__ void vscale(float& a, float s) { a *= s; }
__device__ __forceinline__ void vscale(double& a, double s) { a *= s; }

// unresolved, forward: CTA per pixel group, threads over the nv vectors of a row
template <typename T, typename V>
__global__ void mix_unres_fwd(int32_t G, int64_t nv, const int32_t* __restrict__ gp,
                              const int32_t* __restrict__ gr, const T* __restrict__ inv,
                              const V* __restrict__ y, V* __restrict__ yl) {
    for (int g = blockIdx.x; g < G; g += gridDim.x) {
        const int p0 = gp[g], p1 = gp[g + 1];
        const T s = inv[g];
        for (int64_t c = threadIdx.x; c < nv; c += blockDim.x) {
            V acc = y[(int64_t)gr[p0] * nv + c];
            for (int p = p0 + 1; p < p1; ++p) vadd(acc, y[(int64_t)gr[p] * nv + c]);
            vscale(acc, s);
            yl[(int64_t)g * nv + c] = acc;
        }
    }
}

// unresolved, adjoint: CTA per arm row, the row's group value times 1 / sqrt(count)
template <typename T, typename V>
__global__ void mix_unres_adj(int32_t R, int64_t nv, const int32_t* __restrict__ row_grp,
                              const T* __restrict__ inv, const V* __restrict__ yl,
                              V* __restrict__ y) {
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        const int g = row_grp[r];
        const T s = inv[g];
        for (int64_t c = threadIdx.x; c < nv; c += blockDim.x) {
            V v = yl[(int64_t)g * nv + c];
            vscale(v, s);
            y[(int64_t)r * nv + c] = v;
        }
    }
}

// total flux, pass 1: block b sums rows [b RB, min(R, (b + 1) RB)) in order
// (eight rows' loads issued before their additions)
template <typename V>
__global__ void mix_flux_part(int32_t R, int32_t RB, int64_t nv, const V* __restrict__ y,
                              V* __restrict__ part) {
    const int b = blockIdx.x;
    const int r0 = b * RB, r1 = min(R, r0 + RB);
    for (int64_t c = threadIdx.x; c < nv; c += blockDim.x) {
        V acc = y[(int64_t)r0 * nv + c];
        int r = r0 + 1;
        for (; r + 8 <= r1; r += 8) {
            V v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = y[(int64_t)(r + u) * nv + c];
#pragma unroll
            for (int u = 0; u < 8; ++u) vadd(acc, v[u]);
        }
        for (; r < r1; ++r) vadd(acc, y[(int64_t)r * nv + c]);
        part[(int64_t)b * nv + c] = acc;
    }
}

// total flux, pass 2: warp per value c; lane l sums the blocks b = l, l + 32,
// ... in order, a fixed shuffle tree adds the lanes; times 1 / sqrt(R)
template <typename T>
__global__ void mix_flux_sum(int32_t nb, int64_t ncols, T inv, const T* __restrict__ part,
                             T* __restrict__ yl) {
    const int lane = threadIdx.x & 31;
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= ncols) return;
    T acc = T(0);
    int b = lane;
    for (; b + 32 * 3 < nb; b += 32 * 4) {
        const T v0 = part[(int64_t)b * ncols + c], v1 = part[(int64_t)(b + 32) * ncols + c];
        const T v2 = part[(int64_t)(b + 64) * ncols + c], v3 = part[(int64_t)(b + 96) * ncols + c];
        acc = acc + v0;
        acc = acc + v1;
        acc = acc + v2;
        acc = acc + v3;
    }
    for (; b < nb; b += 32) acc = acc + part[(int64_t)b * ncols + c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = acc + __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) yl[c] = acc * inv;
}

// total flux, adjoint: every row gets the readout times 1 / sqrt(R)
template <typename T, typename V>
__global__ void mix_flux_adj(int32_t R, int64_t nv, T inv, const V* __restrict__ yl,
                             V* __restrict__ y) {
    for (int r = blockIdx.x; r < R; r += gridDim.x)
        for (int64_t c = threadIdx.x; c < nv; c += blockDim.x) {
            V v = yl[c];
            vscale(v, inv);
            y[(int64_t)r * nv + c] = v;
        }
}

// probe responses of the arm's rows for a chunk of ages (Eq. 10-12):
// y[row][f][a] = scale / N_h sum_{e in row} w_e exp(-(t_o(f) - Delta_e + a)^2
// / (2 h^2)), FP64, terms with exponent below -100 dropped (as the probe
// kernel does); ages past `na` in the chunk are written as zero
__device__ __forceinline__ int mix_arm_row(const ArmSeg& s, int row_out) {
    int r = row_out;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i < s.n && r < s.len[i]) return s.begin[i] + r;
        if (i < s.n) r -= s.len[i];
    }
    return -1;
}

template <int NA>
__global__ void mix_probe_rows(const int32_t* __restrict__ row_ptr, const double* __restrict__ delay,
                               const double* __restrict__ weight, ArmSeg seg, int Tn, double t0,
                               double cadence, double inv_2h2, double wscale,
                               const double* __restrict__ ages, int na, double* __restrict__ y) {
    const int64_t n = (int64_t)seg.total * Tn;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ro = (int)(i / Tn), f = (int)(i - (int64_t)ro * Tn);
        const int row = mix_arm_row(seg, ro);
        const double t = t0 + cadence * f;
        double v[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) v[a] = 0.0;
        for (int e = row_ptr[row]; e < row_ptr[row + 1]; ++e) {
            const double tt = t - delay[e];
            const double we = weight[e];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                if (a < na) {
                    const double d = tt + ages[a];
                    const double arg = d * d * inv_2h2;
                    if (arg < 100.0) v[a] += we * exp(-arg);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) y[i * NA + a] = wscale * v[a];
    }
}

// sum over entries i of y[i][a]^2 per age a: block b takes the entries
// [b per_block, (b + 1) per_block), its threads NA ages x (blockDim / NA)
// strided lanes, then a fixed tree over the lanes in shared memory
template <int NA>
__global__ void mix_sumsq_part(int64_t N, int64_t per_block, const double* __restrict__ y,
                               double* __restrict__ part) {
    __shared__ double sh[256];
    const int a = threadIdx.x % NA, lane = threadIdx.x / NA, nl = blockDim.x / NA;
    const int64_t i0 = (int64_t)blockIdx.x * per_block;
    const int64_t i1 = min(N, i0 + per_block);
    double s = 0.0;
    for (int64_t i = i0 + lane; i < i1; i += nl) {
        const double v = y[i * NA + a];
        s += v * v;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = nl / 2; off > 0; off >>= 1) {
        if (lane < off) sh[threadIdx.x] += sh[threadIdx.x + off * NA];
        __syncthreads();
    }
    if (lane == 0) part[(int64_t)blockIdx.x * NA + a] = sh[a];
}

template <int NA>
__global__ void mix_sumsq_final(int nb, const double* __restrict__ part, double* __restrict__ out) {
    const int a = threadIdx.x;
    if (a >= NA) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * NA + a];
    out[a] = s;
}

static int grid_cap(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(n, 1), 65535); }

// the arm's rows grouped by pixel (host build on first use for an arm mask)
rtt_status mix_prepare(rtt_op_s* op, const ArmSeg& seg) {
    // a pixel's rows of different orders lie in different order blocks, so a
    // row shard does not hold whole pixel groups
    RTT_TRY(whole_only(op, "order mixing"));
    auto& m = op->mix;
    if (m.arm_mask == seg.mask && m.grp_ptr) return RTT_OK;
    const int64_t R = op->n_rows, Ra = seg.total;
    std::vector<int32_t> order(R), pixel(R);
    if (cudaMemcpy(order.data(), op->row_order, R * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(pixel.data(), op->row_pixel, R * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("mix: copying the row keys failed");
        return RTT_ECUDA;
    }
    // arm output row -> (pixel, order)
    std::vector<int32_t> rp(Ra), ro(Ra);
    for (int i = 0; i < seg.n; ++i)
        for (int k = 0; k < seg.len[i]; ++k) {
            rp[seg.out_off[i] + k] = pixel[seg.begin[i] + k];
            ro[seg.out_off[i] + k] = order[seg.begin[i] + k];
        }
    std::vector<int32_t> idx(Ra);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
        return rp[a] != rp[b] ? rp[a] < rp[b] : ro[a] < ro[b];
    });
    std::vector<int32_t> gptr{0}, rgrp(Ra);
    std::vector<double> inv64;
    for (int64_t i = 0; i < Ra; ++i) {
        if (i > 0 && rp[idx[i]] != rp[idx[i - 1]]) gptr.push_back((int32_t)i);
        rgrp[idx[i]] = (int32_t)gptr.size() - 1;
    }
    gptr.push_back((int32_t)Ra);
    const int32_t G = (int32_t)gptr.size() - 1;
    inv64.resize(G);
    std::vector<float> inv32(G);
    for (int g = 0; g < G; ++g) {
        inv64[g] = 1.0 / std::sqrt((double)(gptr[g + 1] - gptr[g]));
        inv32[g] = (float)inv64[g];
    }
    cudaDeviceSynchronize();  // the old tables may still be in use by queued work
    for (void* p : {(void*)m.grp_ptr, (void*)m.grp_rows, (void*)m.row_grp, (void*)m.inv32,
                    (void*)m.inv64})
        if (p) cudaFree(p);
    m = rtt_op_s::MixGroups{-1, 0, nullptr, nullptr, nullptr, nullptr, nullptr, m.part, m.part_bytes};
    cudaError_t e = cudaMalloc(&m.grp_ptr, (G + 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m.grp_rows, std::max<int64_t>(Ra, 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m.row_grp, std::max<int64_t>(Ra, 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m.inv32, std::max(G, 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m.inv64, std::max(G, 1) * 8);
    if (e == cudaSuccess) e = cudaMemcpy(m.grp_ptr, gptr.data(), (G + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && Ra) e = cudaMemcpy(m.grp_rows, idx.data(), Ra * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && Ra) e = cudaMemcpy(m.row_grp, rgrp.data(), Ra * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && G) e = cudaMemcpy(m.inv32, inv32.data(), G * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && G) e = cudaMemcpy(m.inv64, inv64.data(), G * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_error("mix: building the pixel groups failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RTT_ENOMEM : RTT_ECUDA;
    }
    m.arm_mask = seg.mask;
    m.n_groups = G;
    return RTT_OK;
}

int64_t mix_out_rows(const rtt_op_s* op, const ArmSeg& seg, int mode) {
    if (seg.total == 0) return 0;
    return mode == RTT_MIX_TOTAL_FLUX ? 1 : op->mix.n_groups;
}

static rtt_status ensure_part(rtt_op_s* op, size_t bytes) {
    auto& m = op->mix;
    if (m.part_bytes >= bytes) return RTT_OK;
    if (m.part) {
        cudaDeviceSynchronize();
        cudaFree(m.part);
        m.part = nullptr;
        m.part_bytes = 0;
    }
    if (cudaMalloc(&m.part, bytes) != cudaSuccess) {
        set_error("mix: total-flux scratch of %zu bytes", bytes);
        return RTT_ENOMEM;
    }
    m.part_bytes = bytes;
    return RTT_OK;
}

template <typename T, typename V>
static rtt_status mix_fwd_v(rtt_op_s* op, const ArmSeg& seg, int mode, const T* y, T* yl, int64_t nv,
                            cudaStream_t st) {
    const V* yv = reinterpret_cast<const V*>(y);
    V* ylv = reinterpret_cast<V*>(yl);
    const int32_t R = seg.total;
    if (R == 0) return RTT_OK;
    if (mode == RTT_MIX_UNRESOLVED) {
        const auto& m = op->mix;
        const T* inv = sizeof(T) == 4 ? (const T*)m.inv32 : (const T*)m.inv64;
        mix_unres_fwd<T, V><<<grid_cap(m.n_groups), 256, 0, st>>>(m.n_groups, nv, m.grp_ptr, m.grp_rows,
                                                                  inv, yv, ylv);
    } else {
        const int32_t RB = std::max<int32_t>(64, (R + 1023) / 1024);
        const int32_t nb = (R + RB - 1) / RB;
        rtt_status s = ensure_part(op, (size_t)nb * nv * sizeof(V));
        if (s != RTT_OK) return s;
        V* part = reinterpret_cast<V*>(op->mix.part);
        mix_flux_part<V><<<nb, 256, 0, st>>>(R, RB, nv, yv, part);
        const int64_t ncols = nv * (int64_t)(sizeof(V) / sizeof(T));
        mix_flux_sum<T><<<(int)((ncols * 32 + 255) / 256), 256, 0, st>>>(
            nb, ncols, (T)(1.0 / std::sqrt((double)R)), reinterpret_cast<const T*>(part), yl);
    }
    return cudaGetLastError() == cudaSuccess ? RTT_OK : RTT_ECUDA;
}

template <typename T, typename V>
static rtt_status mix_adj_v(rtt_op_s* op, const ArmSeg& seg, int mode, const T* yl, T* y, int64_t nv,
                            cudaStream_t st) {
    const V* ylv = reinterpret_cast<const V*>(yl);
    V* yv = reinterpret_cast<V*>(y);
    const int32_t R = seg.total;
    if (R == 0) return RTT_OK;
    if (mode == RTT_MIX_UNRESOLVED) {
        const auto& m = op->mix;
        const T* inv = sizeof(T) == 4 ? (const T*)m.inv32 : (const T*)m.inv64;
        mix_unres_adj<T, V><<<grid_cap(R), 256, 0, st>>>(R, nv, m.row_grp, inv, ylv, yv);
    } else {
        mix_flux_adj<T, V><<<grid_cap(R), 256, 0, st>>>(R, nv, (T)(1.0 / std::sqrt((double)R)), ylv, yv);
    }
    return cudaGetLastError() == cudaSuccess ? RTT_OK : RTT_ECUDA;
}

// y [arm rows][cols] -> yl [mixed rows][cols] (adjoint = false), or back
template <typename T>
rtt_status launch_mix(rtt_op_s* op, const ArmSeg& seg, int mode, const T* in, T* out, int64_t cols,
                      bool adjoint, cudaStream_t st) {
    rtt_status s = mix_prepare(op, seg);
    if (s != RTT_OK) return s;
    constexpr int W = MixVec<T>::W;
    const bool vec = cols % W == 0 && (uintptr_t)in % 16 == 0 && (uintptr_t)out % 16 == 0;
    using V = typename MixVec<T>::V;
    if (adjoint)
        return vec ? mix_adj_v<T, V>(op, seg, mode, in, out, cols / W, st)
                   : mix_adj_v<T, T>(op, seg, mode, in, out, cols, st);
    return vec ? mix_fwd_v<T, V>(op, seg, mode, in, out, cols / W, st)
               : mix_fwd_v<T, T>(op, seg, mode, in, out, cols, st);
}

template rtt_status launch_mix<float>(rtt_op_s*, const ArmSeg&, int, const float*, float*, int64_t,
                                      bool, cudaStream_t);
template rtt_status launch_mix<double>(rtt_op_s*, const ArmSeg&, int, const double*, double*, int64_t,
                                       bool, cudaStream_t);

}  // namespace rtt

using namespace rtt;

static rtt_status mix_args(rtt_op op, int arm_mask, int mode, const void* a, const void* b, int batch,
                           ArmSeg* seg) {
    if (!op || !a || !b || batch < 1 || (mode != RTT_MIX_UNRESOLVED && mode != RTT_MIX_TOTAL_FLUX)) {
        set_error("invalid mix arguments (mode=%d batch=%d)", mode, batch);
        return RTT_EINVAL;
    }
    RTT_TRY(whole_only(op, "order mixing"));
    return make_seg(op, arm_mask, seg);
}

extern "C" rtt_status rtt_mix_rows_count(rtt_op op, int arm_mask, int mode, int64_t* n_out) {
    if (!op || !n_out || (mode != RTT_MIX_UNRESOLVED && mode != RTT_MIX_TOTAL_FLUX)) {
        set_error("invalid mix arguments (mode=%d)", mode);
        return RTT_EINVAL;
    }
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s == RTT_OK) s = mix_prepare(op, seg);
    if (s == RTT_OK) *n_out = mix_out_rows(op, seg, mode);
    return s;
}

template <typename T>
static rtt_status mix_call(rtt_op op, int arm_mask, int mode, const T* in, T* out, int batch, bool adj,
                           void* stream) {
    ArmSeg seg;
    rtt_status s = mix_args(op, arm_mask, mode, in, out, batch, &seg);
    if (s != RTT_OK) return s;
    const int64_t cols = (int64_t)op->time.n_frames * batch;
    s = launch_mix<T>(op, seg, mode, in, out, cols, adj, (cudaStream_t)stream);
    if (s == RTT_ECUDA) set_error("mix: %s", cudaGetErrorString(cudaGetLastError()));
    return s;
}

extern "C" rtt_status rtt_mix_rows(rtt_op op, int arm_mask, int mode, const float* y_dev, float* yl_dev,
                                   int batch, void* stream) {
    return mix_call<float>(op, arm_mask, mode, y_dev, yl_dev, batch, false, stream);
}
extern "C" rtt_status rtt_mix_rows_T(rtt_op op, int arm_mask, int mode, const float* yl_dev, float* y_dev,
                                     int batch, void* stream) {
    return mix_call<float>(op, arm_mask, mode, yl_dev, y_dev, batch, true, stream);
}
extern "C" rtt_status rtt_mix_rows_f64(rtt_op op, int arm_mask, int mode, const double* y_dev,
                                       double* yl_dev, int batch, void* stream) {
    return mix_call<double>(op, arm_mask, mode, y_dev, yl_dev, batch, false, stream);
}
extern "C" rtt_status rtt_mix_rows_T_f64(rtt_op op, int arm_mask, int mode, const double* yl_dev,
                                         double* y_dev, int batch, void* stream) {
    return mix_call<double>(op, arm_mask, mode, yl_dev, y_dev, batch, true, stream);
}

extern "C" rtt_status rtt_probe_info_mix(rtt_op op, int arm_mask, int mode, int n_ages,
                                         const double* ages_host, double h, double* info_host,
                                         void* stream) {
    if (!op || !ages_host || !info_host || n_ages < 1 || n_ages > 4096 || !(h > 0.0) ||
        (mode != RTT_MIX_UNRESOLVED && mode != RTT_MIX_TOTAL_FLUX)) {
        set_error("invalid mixed-probe arguments (mode=%d n_ages=%d h=%g)", mode, n_ages, h);
        return RTT_EINVAL;
    }
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s == RTT_OK) s = mix_prepare(op, seg);
    if (s != RTT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    constexpr int NA = 16;
    const int Tn = op->time.n_frames;
    const int64_t Ra = seg.total, Rl = mix_out_rows(op, seg, mode);
    if (Ra == 0) {
        for (int i = 0; i < n_ages; ++i) info_host[i] = 0.0;
        return RTT_OK;
    }
    const int64_t N = Rl * Tn;  // mixed (row, frame) entries
    const int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (N + 4095) / 4096));
    const int64_t per_block = (N + nb - 1) / nb;
    double *ages = nullptr, *y = nullptr, *yl = nullptr, *part = nullptr, *info = nullptr;
    cudaError_t e = cudaMalloc(&ages, (size_t)n_ages * 8);
    if (e == cudaSuccess) e = cudaMalloc(&y, (size_t)Ra * Tn * NA * 8);
    if (e == cudaSuccess) e = cudaMalloc(&yl, (size_t)std::max<int64_t>(N, 1) * NA * 8);
    if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)nb * NA * 8);
    if (e == cudaSuccess) e = cudaMalloc(&info, NA * 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ages, ages_host, (size_t)n_ages * 8, cudaMemcpyHostToDevice, st);
    const double Nh = std::sqrt(M_PI * (op->grid.r_out * op->grid.r_out - op->grid.r_in * op->grid.r_in) *
                                h * std::sqrt(M_PI));
    for (int c0 = 0; e == cudaSuccess && c0 < n_ages; c0 += NA) {
        const int na = std::min(NA, n_ages - c0);
        mix_probe_rows<NA><<<grid_cap((Ra * Tn + 255) / 256), 256, 0, st>>>(
            op->row_ptr, op->delay, op->weight, seg, Tn, op->time.t0, op->time.cadence,
            1.0 / (2.0 * h * h), op->scale / Nh, ages + c0, na, y);
        e = cudaGetLastError();
        if (e == cudaSuccess &&
            launch_mix<double>(op, seg, mode, y, yl, (int64_t)Tn * NA, false, st) != RTT_OK)
            e = cudaErrorUnknown;
        if (e == cudaSuccess) {
            mix_sumsq_part<NA><<<nb, 256, 0, st>>>(N, per_block, yl, part);
            mix_sumsq_final<NA><<<1, 32, 0, st>>>(nb, part, info);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(info_host + c0, info, (size_t)na * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    for (double* p : {ages, y, yl, part, info})
        if (p) cudaFree(p);
    if (e != cudaSuccess) {
        set_error("mixed probe information: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RTT_ENOMEM : RTT_ECUDA;
    }
    return RTT_OK;
}
