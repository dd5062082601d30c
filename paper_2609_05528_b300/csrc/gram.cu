// Restricted Gram matrix, symmetric eigendecomposition and operational rank
// (Sec. 3.2 Eq. 7, Sec. 4.1 Eq. 21, Sec. 4.4 Eq. 31).
//
//   P = scale * A Q  (rows (row, frame), columns the d class directions)
//   G = P^T P        (d x d, FP64)
//   sigma_i = sqrt(max(lambda_i(G), 0)),  rank = #{sigma_i >= rho}
//
// The Gram is accumulated over row chunks of the operator: for each chunk the
// forward kernel writes P_chunk (FP64) into scratch and a tiled FP64 kernel
// adds P_chunk^T P_chunk.  Partial sums over fixed row splits are reduced in
// a fixed order (deterministic).  The eigendecomposition is a parallel
// cyclic two-sided Jacobi method (round-robin pair ordering) in one CTA.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "rtt_internal.cuh"

namespace rtt {
rtt_status gemm_tn_f64(int64_t k, int m, int n, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int* status, cudaStream_t st);


// dst[n][j] = Q[n][c0 + j], j < w
__global__ void copy_cols(const double* Q, int64_t n, int d, int c0, int w, double* dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * w) return;
    const int64_t row = t / w;
    const int j = (int)(t - row * w);
    dst[t] = Q[row * d + c0 + j];
}

// dst[row][c0 + j] = src[row][j], j < w (a column block into a d-wide matrix)
__global__ void put_cols(const double* src, int64_t n, int d, int c0, int w, double* dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * w) return;
    const int64_t row = t / w;
    const int j = (int)(t - row * w);
    dst[row * d + c0 + j] = src[t];
}

// G <- (G + G^T) / 2
__global__ void symmetrize(double* G, int d) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)d * d) return;
    const int i = (int)(t / d), j = (int)(t - (int64_t)i * d);
    if (i < j) {
        const double v = 0.5 * (G[(int64_t)i * d + j] + G[(int64_t)j * d + i]);
        G[(int64_t)i * d + j] = v;
        G[(int64_t)j * d + i] = v;
    }
}

constexpr int kGT = 32;        // Gram tile edge
constexpr int kGramSplits = 64;  // row splits per chunk (partial sums)

// partial[split][tile][32*32]: sum over the split's rows of P[:, I]^T P[:, J]
__global__ void __launch_bounds__(256) gram_f64_kernel(const double* __restrict__ P, int64_t m,
                                                       int d, int n_tiles_1d,
                                                       const int2* __restrict__ tiles,
                                                       double* __restrict__ partial) {
    __shared__ double sI[kGT][kGT + 1];
    __shared__ double sJ[kGT][kGT + 1];
    const int tile = blockIdx.x;
    const int split = blockIdx.y;
    const int2 tj = tiles[tile];
    const int i0 = tj.x * kGT, j0 = tj.y * kGT;
    const int tid = threadIdx.x;
    // each thread owns 4 entries: rows ti*4.. of the 32x32 tile? use (r, c) = (tid/8*... )
    const int r = tid >> 3;          // 0..31
    const int c0 = (tid & 7) * 4;    // 0..28
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t per = (m + gridDim.y - 1) / gridDim.y;
    const int64_t m_begin = (int64_t)split * per;
    const int64_t m_end = m_begin + per < m ? m_begin + per : m;
    for (int64_t mb = m_begin; mb < m_end; mb += kGT) {
        // load 32 rows x 32 columns for I and J
        for (int idx = tid; idx < kGT * kGT; idx += 256) {
            const int rr = idx >> 5, cc = idx & 31;
            const int64_t row = mb + rr;
            double vi = 0.0, vj = 0.0;
            if (row < m_end) {
                if (i0 + cc < d) vi = P[row * d + i0 + cc];
                if (j0 + cc < d) vj = P[row * d + j0 + cc];
            }
            sI[rr][cc] = vi;
            sJ[rr][cc] = vj;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kGT; ++k) {
            const double a = sI[k][r];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(a, sJ[k][c0 + q], acc[q]);
        }
        __syncthreads();
    }
    double* out = partial + ((int64_t)split * n_tiles_1d * n_tiles_1d + tile) * (kGT * kGT);
    // (tile < number of upper tiles <= n_tiles_1d^2)
#pragma unroll
    for (int q = 0; q < 4; ++q) out[r * kGT + c0 + q] = acc[q];
}

// G[i][j] (+)= sum_split partial; mirrored into the lower triangle.
__global__ void gram_reduce(const double* partial, int n_splits, int n_tiles, const int2* tiles,
                            int d, int accumulate, double* G) {
    const int tile = blockIdx.x;
    const int2 tj = tiles[tile];
    for (int e = threadIdx.x; e < kGT * kGT; e += blockDim.x) {
        const int r = e >> 5, c = e & 31;
        const int i = tj.x * kGT + r, j = tj.y * kGT + c;
        // upper triangle only: each (i, j) and its mirror are owned by one thread
        if (i >= d || j >= d || i > j) continue;
        double s = 0.0;
        for (int sp = 0; sp < n_splits; ++sp)
            s += partial[((int64_t)sp * n_tiles + tile) * (kGT * kGT) + e];
        const double v = accumulate ? G[(int64_t)i * d + j] + s : s;
        G[(int64_t)i * d + j] = v;
        if (i != j) G[(int64_t)j * d + i] = v;
    }
}

// ---------------------------------------------------------------------------
// Parallel cyclic Jacobi (one CTA).  A (n x n, row-major, symmetric) is
// overwritten; V receives the eigenvectors (columns).  A rotation of pair
// (p, q) is skipped when |a_pq| <= eps sqrt(|a_pp a_qq|) (relative
// criterion); the sweep loop ends when a sweep performs no rotation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) jacobi_kernel(double* A_all, double* V_all, int n, int np2,
                                                      int max_sweeps, double eps,
                                                      int* sweeps_all) {
    // one CTA per matrix of the batch
    double* A = A_all + (int64_t)blockIdx.x * n * n;
    double* V = V_all + (int64_t)blockIdx.x * n * n;
    int* sweeps_out = sweeps_all + blockIdx.x;
    extern __shared__ unsigned char jsm[];
    int* perm = reinterpret_cast<int*>(jsm);                  // np2 players
    double* cs = reinterpret_cast<double*>(perm + np2 + (np2 & 1));  // 6 values per pair
    __shared__ int rotated;
    __shared__ double floor_abs;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int half = np2 / 2;
    if (tid == 0) {
        double m = 0.0;
        for (int i = 0; i < n; ++i) m = fmax(m, fabs(A[(int64_t)i * n + i]));
        // couplings below 1e-18 of the largest diagonal cannot move any
        // eigenvalue by more than rounding already does
        floor_abs = 1e-18 * m;
    }
    for (int i = tid; i < n * n; i += nt) V[i] = (i / n == i % n) ? 1.0 : 0.0;
    for (int i = tid; i < np2; i += nt) perm[i] = i;
    __syncthreads();
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < np2 - 1; ++round) {
            // rotation parameters for the round's disjoint pairs
            for (int k = tid; k < half; k += nt) {
                int p = perm[k], q = perm[np2 - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0, tt = 0.0, apq0 = 0.0, app0 = 0.0, aqq0 = 0.0;
                if (q < n) {
                    const double apq = A[(int64_t)p * n + q];
                    const double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
                    if (fabs(apq) > fmax(eps * sqrt(fabs(app * aqq)), floor_abs)) {
                        const double theta = (aqq - app) / (2.0 * apq);
                        const double t = (theta >= 0.0 ? 1.0 : -1.0) /
                                         (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                        tt = t;
                        apq0 = apq;
                        app0 = app;
                        aqq0 = aqq;
                        rotated = 1;
                    }
                }
                cs[6 * k] = c;
                cs[6 * k + 1] = s;
                cs[6 * k + 2] = tt;
                cs[6 * k + 3] = apq0;
                cs[6 * k + 4] = app0;
                cs[6 * k + 5] = aqq0;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int idx = tid; idx < half * n; idx += nt) {
                const int k = idx / n, col = idx - k * n;
                int p = perm[k], q = perm[np2 - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                if (q >= n) continue;
                const double c = cs[6 * k], s = cs[6 * k + 1];
                if (s == 0.0) continue;
                const double ap = A[(int64_t)p * n + col], aq = A[(int64_t)q * n + col];
                A[(int64_t)p * n + col] = c * ap - s * aq;
                A[(int64_t)q * n + col] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int idx = tid; idx < half * n; idx += nt) {
                const int k = idx / n, row = idx - k * n;
                int p = perm[k], q = perm[np2 - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                if (q >= n) continue;
                const double c = cs[6 * k], s = cs[6 * k + 1];
                if (s == 0.0) continue;
                const double ap = A[(int64_t)row * n + p], aq = A[(int64_t)row * n + q];
                A[(int64_t)row * n + p] = c * ap - s * aq;
                A[(int64_t)row * n + q] = s * ap + c * aq;
                const double vp = V[(int64_t)row * n + p], vq = V[(int64_t)row * n + q];
                V[(int64_t)row * n + p] = c * vp - s * vq;
                V[(int64_t)row * n + q] = s * vp + c * vq;
            }
            __syncthreads();
            // the rotated 2x2 block exactly: a_pq = 0, a_pp -= t a_pq, a_qq += t a_pq
            for (int k = tid; k < half; k += nt) {
                int p = perm[k], q = perm[np2 - 1 - k];
                if (p > q) { const int t = p; p = q; q = t; }
                if (q >= n || cs[6 * k + 1] == 0.0) continue;
                const double t = cs[6 * k + 2], apq = cs[6 * k + 3];
                A[(int64_t)p * n + q] = 0.0;
                A[(int64_t)q * n + p] = 0.0;
                A[(int64_t)p * n + p] = cs[6 * k + 4] - t * apq;
                A[(int64_t)q * n + q] = cs[6 * k + 5] + t * apq;
            }
            __syncthreads();
            // round-robin: keep player 0, rotate the others by one
            if (tid == 0) {
                const int last = perm[np2 - 1];
                for (int i = np2 - 1; i > 1; --i) perm[i] = perm[i - 1];
                perm[1] = last;
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) break;
    }
    if (tid == 0) *sweeps_out = sweep;
}

}  // namespace rtt

using namespace rtt;

extern "C" rtt_status rtt_gram(rtt_op op, int arm_mask, const double* Q, int d, double* G,
                               void* stream) {
    if (!op || !Q || !G || d < 1 || d > 4096) {
        set_error("invalid gram arguments (d=%d)", d);
        return RTT_EINVAL;
    }
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s != RTT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int Tn = op->time.n_frames;
    // rows per chunk: P_chunk <= 1 GiB
    const int64_t bytes_per_row = (int64_t)Tn * d * 8;
    int64_t chunk = ((int64_t)1 << 30) / bytes_per_row;
    if (chunk < 1) chunk = 1;
    const int nt = (d + kGT - 1) / kGT;
    std::vector<int2> tiles;
    for (int i = 0; i < nt; ++i)
        for (int j = i; j < nt; ++j) tiles.push_back(make_int2(i, j));
    const int n_tiles = (int)tiles.size();
    double *P = nullptr, *partial = nullptr;
    int2* d_tiles = nullptr;
    const int64_t max_rows = chunk < seg.total ? chunk : (seg.total > 0 ? seg.total : 1);
    cudaError_t e = cudaMalloc(&P, (size_t)max_rows * bytes_per_row);
    // partial sums are indexed [split][ti * nt + tj]: nt * nt slots per split
    if (e == cudaSuccess) e = cudaMalloc(&partial, (size_t)kGramSplits * nt * nt * kGT * kGT * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_tiles, n_tiles * sizeof(int2));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tiles, tiles.data(), n_tiles * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, (size_t)d * d * 8, st);
    int first = 1;
    for (int sg = 0; e == cudaSuccess && sg < seg.n; ++sg) {
        for (int64_t off = 0; e == cudaSuccess && off < seg.len[sg]; off += chunk) {
            const int64_t len = seg.len[sg] - off < chunk ? seg.len[sg] - off : chunk;
            ArmSeg cs{};
            cs.n = 1;
            cs.begin[0] = seg.begin[sg] + (int32_t)off;
            cs.len[0] = (int32_t)len;
            cs.out_off[0] = 0;
            cs.total = (int32_t)len;
            cs.mask = arm_mask;
            e = launch_forward<double>(op, Q, P, d, cs, st);
            if (e != cudaSuccess) break;
            const int64_t m = len * Tn;
            gram_f64_kernel<<<dim3(n_tiles, kGramSplits), 256, 0, st>>>(P, m, d, nt, d_tiles,
                                                                       partial);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
            // the partial array is indexed [split][tile] with n_tiles_1d^2 slots
            gram_reduce<<<n_tiles, 256, 0, st>>>(partial, kGramSplits, nt * nt, d_tiles, d,
                                                 first ? 0 : 1, G);
            e = cudaGetLastError();
            first = 0;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(P);
    cudaFree(partial);
    cudaFree(d_tiles);
    if (e != cudaSuccess) {
        set_error("gram: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RTT_ENOMEM : RTT_ECUDA;
    }
    return RTT_OK;
}

// G = Q^T (A^T (A Q)) through the normal operator, FP64 throughout: the
// contraction runs over the n_nodes * n_hats source coefficients instead of
// the rows * frames data samples (about 18x fewer at kerr256 sizes), which is
// what makes an FP64-accurate Gram affordable on FP64-poor hardware.
static rtt_status gram_normal_impl(rtt_op op, int arm_mask, int mix_mode, const double* Q, int d,
                                   double* G, void* stream) {
    if (!op || !Q || !G || d < 1 || d > 4096) {
        set_error("invalid gram arguments (d=%d)", d);
        return RTT_EINVAL;
    }
    if (mix_mode) RTT_TRY(whole_only(op, "order mixing"));
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s != RTT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int W = 32;  // columns per pass
    const int64_t N = (int64_t)op->n_nodes * op->time.n_hats;
    const int64_t M = (int64_t)seg.total * op->time.n_frames;
    s = ensure_adjoint_scratch(op, W, (int)sizeof(double));
    if (s != RTT_OK) return s;
    double *Qc = nullptr, *Y = nullptr, *Z = nullptr, *YL = nullptr;
    if (mix_mode) {
        s = mix_prepare(op, seg);
        if (s != RTT_OK) return s;
    }
    const int64_t ML = mix_mode ? mix_out_rows(op, seg, mix_mode) * op->time.n_frames : 0;
    cudaError_t e = cudaMalloc(&Qc, (size_t)N * W * 8);
    if (e == cudaSuccess) e = cudaMalloc(&Y, (size_t)(M > 0 ? M : 1) * W * 8);
    if (e == cudaSuccess) e = cudaMalloc(&Z, (size_t)N * W * 8);
    if (e == cudaSuccess && mix_mode) e = cudaMalloc(&YL, (size_t)(ML > 0 ? ML : 1) * W * 8);
    // Z = A^T A Q, column block by column block, gathered into one N x d matrix
    double* Zf = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&Zf, (size_t)N * d * 8);
    for (int c0 = 0; e == cudaSuccess && c0 < d; c0 += W) {
        const int w = d - c0 < W ? d - c0 : W;
        copy_cols<<<(int)((N * w + 255) / 256), 256, 0, st>>>(Q, N, d, c0, w, Qc);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_forward<double>(op, Qc, Y, w, seg, st);
        if (e == cudaSuccess && mix_mode) {
            // Y <- W^T W Y: the mixed arm's data and back (Eq. 4)
            const int64_t cols = (int64_t)op->time.n_frames * w;
            if (launch_mix<double>(op, seg, mix_mode, Y, YL, cols, false, st) != RTT_OK ||
                launch_mix<double>(op, seg, mix_mode, YL, Y, cols, true, st) != RTT_OK)
                e = cudaErrorUnknown;
        }
        if (e == cudaSuccess) e = launch_adjoint<double>(op, Y, Z, w, seg, st);
        if (e == cudaSuccess) {
            put_cols<<<(int)((N * w + 255) / 256), 256, 0, st>>>(Z, N, d, c0, w, Zf);
            e = cudaGetLastError();
        }
    }
    cudaFree(Qc);
    cudaFree(Y);
    cudaFree(Z);
    if (YL) cudaFree(YL);
    // G = Q^T Z on the tensor cores in FP64 accuracy (digit splitting)
    rtt_status gs = RTT_OK;
    if (e == cudaSuccess) gs = gemm_tn_f64(N, d, d, Q, d, Zf, d, G, d, op->dev_status, st);
    if (e == cudaSuccess && gs == RTT_OK) {
        symmetrize<<<(int)(((int64_t)d * d + 255) / 256), 256, 0, st>>>(G, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && gs == RTT_OK) e = cudaStreamSynchronize(st);
    cudaFree(Zf);
    if (gs != RTT_OK) return gs;
    if (e != cudaSuccess) {
        set_error("gram (normal operator): %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RTT_ENOMEM : RTT_ECUDA;
    }
    return RTT_OK;
}

extern "C" rtt_status rtt_gram_normal(rtt_op op, int arm_mask, const double* Q, int d, double* G,
                                      void* stream) {
    return gram_normal_impl(op, arm_mask, 0, Q, d, G, stream);
}

extern "C" rtt_status rtt_gram_normal_mix(rtt_op op, int arm_mask, int mode, const double* Q, int d,
                                          double* G, void* stream) {
    if (mode != RTT_MIX_UNRESOLVED && mode != RTT_MIX_TOTAL_FLUX) {
        set_error("invalid mix mode %d", mode);
        return RTT_EINVAL;
    }
    return gram_normal_impl(op, arm_mask, mode, Q, d, G, stream);
}

extern "C" rtt_status rtt_eig_sym_batched(int n, int batch, double* A, double* evals_host,
                                          double* V, int max_sweeps, int* sweeps_host,
                                          void* stream) {
    if (n < 1 || n > 4096 || batch < 1 || !A || !evals_host || !V || max_sweeps < 1) {
        set_error("invalid eig arguments (n=%d, batch=%d)", n, batch);
        return RTT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int np2 = n + (n & 1);
    int* d_sw = nullptr;
    cudaError_t e = cudaMalloc(&d_sw, 4 * batch);
    const size_t smem = (size_t)(np2 + 2) * 4 + (size_t)(np2 / 2) * 6 * 8 + 16;
    if (e == cudaSuccess && smem > 48 * 1024)
        e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        jacobi_kernel<<<batch, 1024, smem, st>>>(A, V, n, np2, max_sweeps, 2.2e-16, d_sw);
        e = cudaGetLastError();
    }
    std::vector<int> sweeps(batch);
    for (int b = 0; e == cudaSuccess && b < batch; ++b)
        e = cudaMemcpy2DAsync(evals_host + (int64_t)b * n, 8, A + (int64_t)b * n * n,
                              (size_t)(n + 1) * 8, 8, n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sweeps.data(), d_sw, 4 * batch, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_sw);
    if (e != cudaSuccess) {
        set_error("eig: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    bool ok = true;
    for (int b = 0; b < batch; ++b) {
        if (sweeps_host) sweeps_host[b] = sweeps[b];
        ok = ok && sweeps[b] < max_sweeps;
    }
    if (!ok) {
        set_error("Jacobi did not converge in %d sweeps", max_sweeps);
        return RTT_ENOTCONVERGED;
    }
    return RTT_OK;
}

extern "C" rtt_status rtt_eig_sym(int n, double* A, double* evals_host, double* V, int max_sweeps,
                                  int* sweeps_host, void* stream) {
    return rtt_eig_sym_batched(n, 1, A, evals_host, V, max_sweeps, sweeps_host, stream);
}
