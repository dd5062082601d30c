// Restricted Gram of a separable representation class without forming P
// (Sec. 3.2 Eq. 7 and Eq. 8, Sec. 4.1 Eq. 21, classes of Sec. 6 and Sec. 7).
//
// For the classes synthesised by rtt_synth_class, Q[(s, k)][(a b) 8 + c] =
// R_a(i_s) Phi_b(j_s) tau_c(k), and the bilinear interpolation of a separable
// nodal function is separable.  For ray e of a data row,
//   s_e[a b]  = sum over its 4 corners of W_corner R_a(i) Phi_b(j)   (28 values)
//   h_c(e, f) = (1 - fr) tau_c(k0) + fr tau_c(k0 + 1)                 (the hat
//               interpolation of tau_c at the frame's exact hat coordinate)
// so that P[(row, f)][(a b, c)] = sum_{e in row} s_e[a b] h_c(e, f), and
//   G = P^T P = sum_rows sum_{e, e' in row} (s_e s_e'^T) (x) C_row[(e, c), (e', c')],
//   C_row[(e, c), (e', c')] = sum_f h_c(e, f) h_c'(e', f).
// This needs about 7x fewer FP64 operations than the normal-operator form
// (no 224-column applies, no 524288 x 224 x 224 GEMM) -- FP64 is the scarce
// unit on this GPU.  Everything is FP64; partial tiles are reduced in a fixed
// order (deterministic).  Rows with more than kMaxRayRow rays are not
// handled (the caller falls back to the normal-operator Gram).
#include <cub/cub.cuh>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rtt_internal.cuh"

namespace rtt {

constexpr int kMaxRayRow = 4;    // rays per data row handled here (2x2 sub-rays)
constexpr int kCD = 224;         // class dimension
constexpr int kTile = 56;        // G tile edge: 7 spatial functions x 8 temporal
constexpr int kTilesPerDim = 4;  // 224 / 56
constexpr int kTileThreads = 256;
constexpr int kTileRegs = (kTile * kTile + kTileThreads - 1) / kTileThreads;  // 13
constexpr int kRowChunks = 148;  // row chunks of the tile pass (partial sums)

// 1D class factors, the formulas of the synthesis kernel
__global__ void class_factor_kernel(int n_r, int n_phi, int K, double t_end, double hat_step,
                                    int kind, double* Rt, double* Pt, double* Tt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_r * 4) {
        const int ir = t / 4, i = t % 4;
        const double s = (double)ir / (double)(n_r - 1);
        const double binom[4] = {1.0, 3.0, 3.0, 1.0};
        double R = binom[i];
        for (int q = 0; q < i; ++q) R *= s;
        for (int q = 0; q < 3 - i; ++q) R *= (1.0 - s);
        Rt[t] = R;
    }
    if (t < n_phi * 7) {
        const int jp = t / 7, l = t % 7;
        const double phi = 6.283185307179586476925286766559 * (double)jp / (double)n_phi;
        double Ph = 1.0;
        if (l > 0) {
            const int mm = (l + 1) / 2;
            Ph = (l & 1) ? cos(mm * phi) : sin(mm * phi);
        }
        Pt[t] = Ph;
    }
    if (t < K * 8) {
        const int k = t / 8, m = t % 8;
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
        Tt[t] = tau;
    }
}

__device__ __forceinline__ int arm_row_of(const ArmSeg& s, int row_out) {
    int r = row_out;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i < s.n && r < s.len[i]) return s.begin[i] + r;
        if (i < s.n) r -= s.len[i];
    }
    return -1;
}

// C block sizes (8 n)^2 per arm row and the too-many-rays flag
__global__ void class_row_sizes(const int32_t* row_ptr, ArmSeg seg, int64_t* sizes, int* flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= seg.total) return;
    const int row = arm_row_of(seg, i);
    const int n = row_ptr[row + 1] - row_ptr[row];
    if (n > kMaxRayRow) atomicOr(flag, 1);
    sizes[i] = (int64_t)64 * n * n;
}

// s_e[a b] for every ray of the arm's rows (ray-indexed, 28 doubles each)
__global__ void class_ray_space(const int32_t* row_ptr, ArmSeg seg, const int32_t* node00,
                                const int32_t* node01, const double* W64, int n_phi,
                                const double* Rt, const double* Pt, double* S) {
    const int i = blockIdx.x;  // arm row
    if (i >= seg.total) return;
    const int row = arm_row_of(seg, i);
    for (int e = row_ptr[row]; e < row_ptr[row + 1]; ++e) {
        const int n00 = node00[e], n01 = node01[e];
        const int i0 = n00 / n_phi, j0 = n00 - i0 * n_phi, j1 = n01 - i0 * n_phi;
        for (int t = threadIdx.x; t < 28; t += blockDim.x) {
            const int a = t / 7, b = t % 7;
            // corners (i0 j0), (i0+1 j0), (i0 j1), (i0+1 j1), as in W64
            const double v = W64[4 * (int64_t)e + 0] * Rt[i0 * 4 + a] * Pt[j0 * 7 + b] +
                              W64[4 * (int64_t)e + 1] * Rt[(i0 + 1) * 4 + a] * Pt[j0 * 7 + b] +
                              W64[4 * (int64_t)e + 2] * Rt[i0 * 4 + a] * Pt[j1 * 7 + b] +
                              W64[4 * (int64_t)e + 3] * Rt[(i0 + 1) * 4 + a] * Pt[j1 * 7 + b];
            S[(int64_t)e * 28 + t] = v;
        }
    }
}

constexpr int kCFrames = 32;  // frames per shared-memory chunk of h

// C_row for every arm row: one CTA per row, (8n)^2 entries over 256 threads
__global__ void __launch_bounds__(256)
class_row_C(const int32_t* row_ptr, ArmSeg seg, const int32_t* K0, const int32_t* F0,
            const double* F64, int64_t D, int Tn, int K, const double* Tt, const int64_t* off,
            double* C) {
    __shared__ double h[kMaxRayRow * 8][kCFrames + 1];
    const int i = blockIdx.x;
    if (i >= seg.total) return;
    const int row = arm_row_of(seg, i);
    const int e0 = row_ptr[row], n = row_ptr[row + 1] - e0;
    const int m = 8 * n;  // C is m x m
    const int nent = m * m;
    constexpr int kCRegs = (kMaxRayRow * 8) * (kMaxRayRow * 8) / 256;  // C entries per thread
    double acc[kCRegs];
#pragma unroll
    for (int j = 0; j < kCRegs; ++j) acc[j] = 0.0;
    for (int f0 = 0; f0 < Tn; f0 += kCFrames) {
        // h[(e, c)][fl] at frame f0 + fl (0 beyond the last frame)
        for (int t = threadIdx.x; t < m * kCFrames; t += blockDim.x) {
            const int p = t / kCFrames, fl = t - p * kCFrames;
            const int e = e0 + p / 8, c = p % 8;
            const int f = f0 + fl;
            double v = 0.0;
            if (f < Tn) {
                const int64_t U = (int64_t)K0[e] * kFracOne + (int64_t)F0[e] - (int64_t)f * D;
                const int k0 = (int)(U >> kFracBits);
                // exact hat fraction of the frame (as the FP64 applies take it)
                double fr = F64[e] - (double)(((int64_t)f * D) & kFracMask) * (1.0 / (double)kFracOne);
                if (fr < 0.0) fr += 1.0;
                const double t0 = (k0 >= 0 && k0 < K) ? Tt[k0 * 8 + c] : 0.0;
                const double t1 = (k0 + 1 >= 0 && k0 + 1 < K) ? Tt[(k0 + 1) * 8 + c] : 0.0;
                v = (1.0 - fr) * t0 + fr * t1;
            }
            h[p][fl] = v;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kCRegs; ++j) {
            const int idx = threadIdx.x + 256 * j;
            if (idx < nent) {
                const int p = idx / m, q = idx - p * m;
                double a = acc[j];
                for (int fl = 0; fl < kCFrames; ++fl) a = fma(h[p][fl], h[q][fl], a);
                acc[j] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kCRegs; ++j) {
        const int idx = threadIdx.x + 256 * j;
        if (idx < nent) C[off[i] + idx] = acc[j];
    }
}

// upper tiles (ti <= tj) of G, partial sums over a chunk of arm rows
__device__ __forceinline__ void tile_pair(int t, int& ti, int& tj) {
    int k = t;
    for (ti = 0; ti < kTilesPerDim; ++ti) {
        const int len = kTilesPerDim - ti;
        if (k < len) {
            tj = ti + k;
            return;
        }
        k -= len;
    }
    ti = tj = 0;
}

// acc += the (ti, tj) tile of sum over arm rows [r_begin, r_end) of
// (s_e s_e'^T) (x) C_row; the row's C block starts at C + off[arm row] (the
// C of the arm's rows) or C + off[operator row] (the C of all rows)
__device__ __forceinline__ void class_tile_rows(const int32_t* row_ptr, const ArmSeg& seg, const double* S,
                                                const int64_t* off, bool off_by_row, const double* C,
                                                int r_begin, int r_end, int ti, int tj, double* acc,
                                                double (*Cs)[kMaxRayRow * 8 + 1], double (*Ys)[kTile + 1],
                                                double (*sI)[7], double (*sJ)[7]) {
    for (int i = r_begin; i < r_end; ++i) {
        const int row = arm_row_of(seg, i);
        const int e0 = row_ptr[row], n = row_ptr[row + 1] - e0;
        const int m = 8 * n;
        const int64_t o = off[off_by_row ? row : i];
        for (int t = threadIdx.x; t < n * 7; t += blockDim.x) {
            const int e = t / 7, l = t % 7;
            sI[e][l] = S[(int64_t)(e0 + e) * 28 + ti * 7 + l];
            sJ[e][l] = S[(int64_t)(e0 + e) * 28 + tj * 7 + l];
        }
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            const int p = t / m, q = t - p * m;
            Cs[p][q] = C[o + t];
        }
        __syncthreads();
        // Y[(e, c)][(l', c')] = sum_e' sJ[e'][l'] C[(e, c)][(e', c')]
        for (int t = threadIdx.x; t < m * kTile; t += blockDim.x) {
            const int p = t / kTile, col = t - p * kTile;
            const int l2 = col / 8, c2 = col % 8;
            double y = 0.0;
            for (int e2 = 0; e2 < n; ++e2) y = fma(sJ[e2][l2], Cs[p][e2 * 8 + c2], y);
            Ys[p][col] = y;
        }
        __syncthreads();
        // G[(l, c)][(l', c')] += sum_e sI[e][l] Y[(e, c)][(l', c')]
#pragma unroll
        for (int j = 0; j < kTileRegs; ++j) {
            const int idx = threadIdx.x + kTileThreads * j;
            if (idx < kTile * kTile) {
                const int r = idx / kTile, col = idx - r * kTile;
                const int l = r / 8, c = r % 8;
                double a = acc[j];
                for (int e = 0; e < n; ++e) a = fma(sI[e][l], Ys[e * 8 + c][col], a);
                acc[j] = a;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kTileThreads)
class_gram_tiles(const int32_t* row_ptr, ArmSeg seg, const double* S, const int64_t* off,
                 const double* C, double* partial) {
    constexpr int NT = kTilesPerDim * (kTilesPerDim + 1) / 2;  // 10
    __shared__ double Cs[kMaxRayRow * 8][kMaxRayRow * 8 + 1];
    __shared__ double Ys[kMaxRayRow * 8][kTile + 1];
    __shared__ double sI[kMaxRayRow][7], sJ[kMaxRayRow][7];
    const int tile = blockIdx.x % NT, chunk = blockIdx.x / NT;
    int ti, tj;
    tile_pair(tile, ti, tj);
    const int rows_per = (seg.total + kRowChunks - 1) / kRowChunks;
    const int r_begin = chunk * rows_per, r_end = min(seg.total, r_begin + rows_per);
    double acc[kTileRegs];
#pragma unroll
    for (int j = 0; j < kTileRegs; ++j) acc[j] = 0.0;
    class_tile_rows(row_ptr, seg, S, off, false, C, r_begin, r_end, ti, tj, acc, Cs, Ys, sI, sJ);
#pragma unroll
    for (int j = 0; j < kTileRegs; ++j) {
        const int idx = threadIdx.x + kTileThreads * j;
        if (idx < kTile * kTile)
            partial[((int64_t)chunk * NT + tile) * kTile * kTile + idx] = acc[j];
    }
}

// ---- the class Grams of many (operator, arm) jobs: one launch over the
// flattened (job, row chunk, tile) items, one reduce over (job, entry)
struct ClassJob {
    const int32_t* row_ptr;
    ArmSeg seg;
    const double* S;      // the operator's ray space values
    const int64_t* off;   // C block offset of every operator row
    const double* C;      // C blocks of all operator rows
    int item0, n_chunks, rows_per_chunk;
    double* G;            // 224 x 224 output
};

__global__ void __launch_bounds__(kTileThreads)
class_gram_tiles_multi(const ClassJob* __restrict__ jobs, int n_jobs, double* partial) {
    constexpr int NT = kTilesPerDim * (kTilesPerDim + 1) / 2;
    __shared__ double Cs[kMaxRayRow * 8][kMaxRayRow * 8 + 1];
    __shared__ double Ys[kMaxRayRow * 8][kTile + 1];
    __shared__ double sI[kMaxRayRow][7], sJ[kMaxRayRow][7];
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].item0 <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ClassJob& J = jobs[lo];
    const int local = (int)blockIdx.x - J.item0;
    const int chunk = local / NT, tile = local - chunk * NT;
    int ti, tj;
    tile_pair(tile, ti, tj);
    const int r_begin = chunk * J.rows_per_chunk;
    const int r_end = min(J.seg.total, r_begin + J.rows_per_chunk);
    double acc[kTileRegs];
#pragma unroll
    for (int j = 0; j < kTileRegs; ++j) acc[j] = 0.0;
    class_tile_rows(J.row_ptr, J.seg, J.S, J.off, true, J.C, r_begin, r_end, ti, tj, acc, Cs, Ys, sI, sJ);
#pragma unroll
    for (int j = 0; j < kTileRegs; ++j) {
        const int idx = threadIdx.x + kTileThreads * j;
        if (idx < kTile * kTile) partial[(int64_t)blockIdx.x * kTile * kTile + idx] = acc[j];
    }
}

// G_j from its chunks' tiles, chunks in order; lower tiles mirrored, diagonal
// tiles symmetrised (as class_gram_reduce)
__global__ void class_gram_reduce_multi(const ClassJob* __restrict__ jobs, const double* partial) {
    constexpr int NT = kTilesPerDim * (kTilesPerDim + 1) / 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kCD * kCD) return;
    const ClassJob& J = jobs[blockIdx.y];
    const int gi = t / kCD, gj = t - gi * kCD;
    auto sum_at = [&](int a, int b) {
        const int ti = a / kTile, tj = b / kTile;  // requires ti <= tj
        int tile = 0;
        for (int x = 0; x < ti; ++x) tile += kTilesPerDim - x;
        tile += tj - ti;
        const int idx = (a - ti * kTile) * kTile + (b - tj * kTile);
        double v = 0.0;
        for (int ch = 0; ch < J.n_chunks; ++ch)
            v += partial[((int64_t)J.item0 + (int64_t)ch * NT + tile) * kTile * kTile + idx];
        return v;
    };
    const int ti = gi / kTile, tj = gj / kTile;
    double v;
    if (ti < tj) v = sum_at(gi, gj);
    else if (ti > tj) v = sum_at(gj, gi);
    else v = 0.5 * (sum_at(gi, gj) + sum_at(gj, gi));
    J.G[t] = v;
}

// G from the partial tiles: chunks summed in order; lower tiles mirrored,
// diagonal tiles symmetrised ((G + G^T) / 2, as the other Gram paths do)
__global__ void class_gram_reduce(const double* partial, double* G) {
    constexpr int NT = kTilesPerDim * (kTilesPerDim + 1) / 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kCD * kCD) return;
    const int gi = t / kCD, gj = t - gi * kCD;
    auto sum_at = [&](int a, int b) {
        const int ti = a / kTile, tj = b / kTile;  // requires ti <= tj
        int tile = 0;
        for (int x = 0; x < ti; ++x) tile += kTilesPerDim - x;
        tile += tj - ti;
        const int idx = (a - ti * kTile) * kTile + (b - tj * kTile);
        double v = 0.0;
        for (int ch = 0; ch < kRowChunks; ++ch) v += partial[((int64_t)ch * NT + tile) * kTile * kTile + idx];
        return v;
    };
    const int ti = gi / kTile, tj = gj / kTile;
    double v;
    if (ti < tj) v = sum_at(gi, gj);
    else if (ti > tj) v = sum_at(gj, gi);
    else v = 0.5 * (sum_at(gi, gj) + sum_at(gj, gi));
    G[t] = v;
}

// ---- batched class Grams: per operator the factor tables, the ray-space
// values and the C blocks of all its rows are built once (create); a run is
// two launches for every (operator, arm) job together
struct ClassOpTables {
    double *Rt = nullptr, *Pt = nullptr, *Tt = nullptr, *S = nullptr, *C = nullptr;
    int64_t* off = nullptr;  // [rows + 1]
};

struct ClassPlan {
    std::vector<ClassOpTables> tables;
    ClassJob* jobs = nullptr;
    double* partial = nullptr;
    int n_jobs = 0, n_items = 0;
};

void class_plan_destroy(ClassPlan* cp) {
    if (!cp) return;
    for (auto& t : cp->tables) {
        void* ps[] = {t.Rt, t.Pt, t.Tt, t.S, t.C, t.off};
        for (void* q : ps) cudaFree(q);
    }
    cudaFree(cp->jobs);
    cudaFree(cp->partial);
    delete cp;
}

// tables of one operator for class `kind` over all its rows (synchronises
// `st`); RTT_ESTATE if a row has more rays than the class path handles
static rtt_status class_op_tables(const rtt_op_s* op, int kind, ClassOpTables* t, cudaStream_t st) {
    ArmSeg all;
    RTT_TRY(make_seg(op, 7, &all));
    const int n_r = op->grid.n_r, n_phi = op->grid.n_phi, K = op->time.n_hats;
    const int64_t R = all.total;
    int* flag = nullptr;
    int64_t* sizes = nullptr;
    void* tmp = nullptr;
    auto fail = [&](rtt_status s, const char* what) {
        cudaFree(flag);
        cudaFree(sizes);
        cudaFree(tmp);
        set_error("class plan: %s", what);
        return s;
    };
    if (cudaMalloc(&t->Rt, sizeof(double) * n_r * 4) != cudaSuccess ||
        cudaMalloc(&t->Pt, sizeof(double) * n_phi * 7) != cudaSuccess ||
        cudaMalloc(&t->Tt, sizeof(double) * K * 8) != cudaSuccess ||
        cudaMalloc(&t->S, sizeof(double) * (op->n_rays > 0 ? op->n_rays : 1) * 28) != cudaSuccess ||
        cudaMalloc(&t->off, sizeof(int64_t) * (R + 1)) != cudaSuccess ||
        cudaMalloc(&sizes, sizeof(int64_t) * (R + 1)) != cudaSuccess || cudaMalloc(&flag, sizeof(int)) != cudaSuccess)
        return fail(RTT_ENOMEM, "table allocation failed");
    const int nf = std::max(std::max(n_r * 4, n_phi * 7), K * 8);
    class_factor_kernel<<<(nf + 255) / 256, 256, 0, st>>>(n_r, n_phi, K, op->time.t_end, op->time.hat_step,
                                                          kind, t->Rt, t->Pt, t->Tt);
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    cudaMemsetAsync(sizes, 0, sizeof(int64_t) * (R + 1), st);
    if (R > 0) class_row_sizes<<<(int)((R + 255) / 256), 256, 0, st>>>(op->row_ptr, all, sizes, flag);
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, sizes, t->off, R + 1, st);
    if (cudaMalloc(&tmp, tb + 16) != cudaSuccess) return fail(RTT_ENOMEM, "scan scratch allocation failed");
    cub::DeviceScan::ExclusiveSum(tmp, tb, sizes, t->off, R + 1, st);
    int flag_h = 0;
    int64_t total = 0;
    cudaMemcpyAsync(&flag_h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&total, t->off + R, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(RTT_ECUDA, "table kernels failed");
    if (flag_h) return fail(RTT_ESTATE, "a data row has more rays than the class path handles");
    if (cudaMalloc(&t->C, sizeof(double) * (total > 0 ? total : 1)) != cudaSuccess)
        return fail(RTT_ENOMEM, "C allocation failed");
    if (R > 0) {
        class_ray_space<<<(unsigned)R, 32, 0, st>>>(op->row_ptr, all, op->node00, op->node01, op->W64, n_phi,
                                                     t->Rt, t->Pt, t->S);
        class_row_C<<<(unsigned)R, 256, 0, st>>>(op->row_ptr, all, op->K0, op->F0, op->F64, op->frame_D,
                                                op->time.n_frames, K, t->Tt, t->off, t->C);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return fail(RTT_ECUDA, "class tables failed");
    cudaFree(flag);
    cudaFree(sizes);
    cudaFree(tmp);
    return RTT_OK;
}

rtt_status class_plan_create(const rtt_op_s* const* ops, int n_ops, const int* job_op, const ArmSeg* segs,
                             int n_jobs, int kind, double* G, cudaStream_t st, ClassPlan** out) {
    *out = nullptr;
    ClassPlan* cp = new (std::nothrow) ClassPlan();
    if (!cp) {
        set_error("class plan: host allocation failed");
        return RTT_ENOMEM;
    }
    cp->tables.resize(n_ops);
    for (int g = 0; g < n_ops; ++g) {
        if (ops[g]->time.n_hats < 2) {
            class_plan_destroy(cp);
            set_error("class plan: the class Gram needs at least 2 hats");
            return RTT_EINVAL;
        }
        const rtt_status s = class_op_tables(ops[g], kind, &cp->tables[g], st);
        if (s != RTT_OK) {
            class_plan_destroy(cp);
            return s;
        }
    }
    // rows per chunk: the whole list in about 8 waves of 148 chunk-tiles
    int64_t total_rows = 0;
    for (int j = 0; j < n_jobs; ++j) total_rows += segs[j].total;
    int rpc = (int)((total_rows + 1183) / 1184);
    if (rpc < 64) rpc = 64;
    constexpr int NT = kTilesPerDim * (kTilesPerDim + 1) / 2;
    std::vector<ClassJob> jobs(n_jobs);
    int items = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const rtt_op_s* op = ops[job_op[j]];
        const ClassOpTables& t = cp->tables[job_op[j]];
        ClassJob& J = jobs[j];
        J.row_ptr = op->row_ptr;
        J.seg = segs[j];
        J.S = t.S;
        J.off = t.off;
        J.C = t.C;
        J.rows_per_chunk = rpc;
        J.n_chunks = segs[j].total > 0 ? (segs[j].total + rpc - 1) / rpc : 0;
        J.item0 = items;
        J.G = G + (size_t)j * kCD * kCD;
        items += J.n_chunks * NT;
    }
    cp->n_jobs = n_jobs;
    cp->n_items = items;
    if (cudaMalloc(&cp->jobs, sizeof(ClassJob) * n_jobs) != cudaSuccess ||
        cudaMalloc(&cp->partial, sizeof(double) * ((size_t)(items > 0 ? items : 1)) * kTile * kTile) != cudaSuccess ||
        cudaMemcpy(cp->jobs, jobs.data(), sizeof(ClassJob) * n_jobs, cudaMemcpyHostToDevice) != cudaSuccess) {
        class_plan_destroy(cp);
        set_error("class plan: device allocation failed");
        return RTT_ENOMEM;
    }
    *out = cp;
    return RTT_OK;
}

cudaError_t class_plan_run(ClassPlan* cp, cudaStream_t st) {
    if (cp->n_items > 0) class_gram_tiles_multi<<<cp->n_items, kTileThreads, 0, st>>>(cp->jobs, cp->n_jobs, cp->partial);
    class_gram_reduce_multi<<<dim3((kCD * kCD + 255) / 256, cp->n_jobs), 256, 0, st>>>(cp->jobs, cp->partial);
    return cudaGetLastError();
}

}  // namespace rtt

using namespace rtt;

namespace {

struct ScratchList {
    std::vector<void*> p;
    ~ScratchList() {
        for (void* q : p) cudaFree(q);
    }
    template <typename T>
    bool get(T** out, size_t n) {
        void* q = nullptr;
        if (cudaMalloc(&q, (n > 0 ? n : 1) * sizeof(T)) != cudaSuccess) return false;
        p.push_back(q);
        *out = (T*)q;
        return true;
    }
};

}  // namespace

extern "C" rtt_status rtt_gram_class(rtt_op op, int arm_mask, int kind, double* G, void* stream) {
    if (!op || !G || (kind != RTT_CLASS_S224 && kind != RTT_CLASS_L224)) {
        set_error("invalid class Gram arguments (kind=%d)", kind);
        return RTT_EINVAL;
    }
    if (op->time.n_hats < 2) {
        set_error("class Gram needs at least 2 hats");
        return RTT_EINVAL;
    }
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s != RTT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
#define GC_CUDA(x)                                                                   \
    do {                                                                             \
        cudaError_t _e = (x);                                                        \
        if (_e != cudaSuccess) {                                                     \
            set_error("class Gram: %s (%s:%d)", cudaGetErrorString(_e), __FILE__, __LINE__); \
            return RTT_ECUDA;                                                        \
        }                                                                            \
    } while (0)
    if (seg.total == 0) {
        GC_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * kCD * kCD, st));
        return RTT_OK;
    }
    const int n_r = op->grid.n_r, n_phi = op->grid.n_phi, K = op->time.n_hats;
    ScratchList sc;
    double *Rt, *Pt, *Tt, *S, *C, *partial;
    int64_t *sizes, *off;
    int* flag;
    if (!sc.get(&Rt, n_r * 4) || !sc.get(&Pt, n_phi * 7) || !sc.get(&Tt, K * 8) ||
        !sc.get(&sizes, (size_t)seg.total + 1) || !sc.get(&off, (size_t)seg.total + 1) ||
        !sc.get(&flag, 1) || !sc.get(&S, (size_t)op->n_rays * 28) ||
        !sc.get(&partial, (size_t)kRowChunks * 10 * kTile * kTile)) {
        set_error("class Gram: scratch allocation failed");
        return RTT_ENOMEM;
    }
    const int nf = (n_r * 4 > n_phi * 7 ? n_r * 4 : n_phi * 7) > K * 8
                       ? (n_r * 4 > n_phi * 7 ? n_r * 4 : n_phi * 7)
                       : K * 8;
    class_factor_kernel<<<(nf + 255) / 256, 256, 0, st>>>(n_r, n_phi, K, op->time.t_end,
                                                          op->time.hat_step, kind, Rt, Pt, Tt);
    GC_CUDA(cudaGetLastError());
    GC_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    GC_CUDA(cudaMemsetAsync(sizes, 0, sizeof(int64_t) * ((size_t)seg.total + 1), st));
    class_row_sizes<<<(seg.total + 255) / 256, 256, 0, st>>>(op->row_ptr, seg, sizes, flag);
    GC_CUDA(cudaGetLastError());
    size_t tb = 0;
    GC_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, sizes, off, seg.total + 1, st));
    void* tmp = nullptr;
    if (!sc.get((unsigned char**)&tmp, tb)) {
        set_error("class Gram: scan scratch allocation failed");
        return RTT_ENOMEM;
    }
    GC_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tb, sizes, off, seg.total + 1, st));
    int flag_h = 0;
    int64_t total_h = 0;
    GC_CUDA(cudaMemcpyAsync(&flag_h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    GC_CUDA(cudaMemcpyAsync(&total_h, off + seg.total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GC_CUDA(cudaStreamSynchronize(st));
    if (flag_h) {
        set_error("class Gram: a data row has more than %d rays", kMaxRayRow);
        return RTT_ESTATE;
    }
    if (!sc.get(&C, (size_t)total_h)) {
        set_error("class Gram: %lld-entry C scratch allocation failed", (long long)total_h);
        return RTT_ENOMEM;
    }
    class_ray_space<<<seg.total, 32, 0, st>>>(op->row_ptr, seg, op->node00, op->node01, op->W64,
                                             n_phi, Rt, Pt, S);
    GC_CUDA(cudaGetLastError());
    class_row_C<<<seg.total, 256, 0, st>>>(op->row_ptr, seg, op->K0, op->F0, op->F64, op->frame_D,
                                          op->time.n_frames, K, Tt, off, C);
    GC_CUDA(cudaGetLastError());
    class_gram_tiles<<<kRowChunks * 10, kTileThreads, 0, st>>>(op->row_ptr, seg, S, off, C, partial);
    GC_CUDA(cudaGetLastError());
    class_gram_reduce<<<(kCD * kCD + 255) / 256, 256, 0, st>>>(partial, G);
    GC_CUDA(cudaGetLastError());
    GC_CUDA(cudaStreamSynchronize(st));  // scratch is freed on return
#undef GC_CUDA
    return RTT_OK;
}
