// Held-out estimators (Sec. 9): ridge / Tikhonov by batched conjugate
// gradients and truncated SVD in a representation class.
//
// Ridge: (A^T A + lambda I) x = A^T d for n_rhs data columns times n_lambda
// regularisation values, all in one batch (column c = rhs * n_lambda + l),
// by conjugate gradients preconditioned with M = diag(D) + lambda, D the
// ray-level diagonal of A^T A (below).  Vectors and applies are FP32;
// per-column dot products accumulate in FP64 in a fixed order; every
// `refresh_every` iterations, and at the end, the residual is recomputed in
// FP64 (FP64 applies on an FP64 copy of x), which keeps the FP32 recurrence
// from drifting and gives the reported residual.
// TSVD: x = Q V_r L_r^{-1} V_r^T Q^T A^T d with (V, L) the eigenpairs of the
// restricted Gram (Eq. 31), FP64, plain GEMMs through cuBLAS.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "kern_common.cuh"

namespace rtt {
rtt_status gemm_tn_f64(int64_t k, int m, int n, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int* status, cudaStream_t st);

// out (cols x rows) = in^T, in: rows x cols row-major
__global__ void transpose_kernel(const double* __restrict__ in, int64_t rows, int cols, double* out) {
    __shared__ double t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int64_t r = r0 + j;
        const int c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[j][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int c = c0 + j;
        const int64_t r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(int64_t)c * rows + r] = t[threadIdx.x][j];
    }
}


// Ray-level diagonal of A^T A for the preconditioner: for coefficient
// (node s, hat k), the sum over the rays of the arm whose stencil touches s of
// W_{e,c}^2 sum_f h_e(f, k)^2, c the corner of e at s and h_e(f, k) the hat
// weight of frame f (the cross terms between rays of one data row are left
// out; the preconditioner only sets the convergence rate, never the
// solution).  One thread per (s, k) walks the rays of the (at most four)
// cells around s in the cell-ordered table: a fixed order, deterministic.
__global__ void ridge_diag_kernel(const int32_t* __restrict__ cell_ptr, const int32_t* __restrict__ c_row,
                                  const int32_t* __restrict__ c_K0, const double* __restrict__ c_F64,
                                  const double* __restrict__ c_W64, ArmSeg seg, int n_r, int n_phi, int K,
                                  int Tn, double delta, double* __restrict__ D) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_r * n_phi * K) return;
    const int s = (int)(t / K), k = (int)(t - (int64_t)s * K);
    const int i = s / n_phi, j = s - i * n_phi;
    const int jm = (j + n_phi - 1) % n_phi;
    // (cell i0, j0; corner of s in that cell): corners ordered (i0 j0),
    // (i0+1 j0), (i0 j1), (i0+1 j1)
    const int ci[4] = {i, i - 1, i, i - 1}, cj[4] = {j, j, jm, jm}, corner[4] = {0, 1, 2, 3};
    double acc = 0.0;
    for (int q = 0; q < 4; ++q) {
        if (ci[q] < 0 || ci[q] > n_r - 2) continue;
        const int cell = ci[q] * n_phi + cj[q];
        for (int p = cell_ptr[cell]; p < cell_ptr[cell + 1]; ++p) {
            if (seg_out_row(seg, c_row[p]) < 0) continue;
            const double w = c_W64[4 * (int64_t)p + corner[q]];
            // frames with |u0 - f delta - k| < 1, u0 = K0 + F
            const double u0 = (double)c_K0[p] + c_F64[p];
            const double fl = floor((u0 - k - 1.0) / delta);
            if (fl >= (double)Tn) continue;
            const int f0 = fl < 0.0 ? 0 : (int)fl;
            double h2 = 0.0;
            for (int f = f0; f < Tn; ++f) {
                const double x = u0 - f * delta - k;
                if (x <= -1.0) break;
                const double hw = 1.0 - fabs(x);
                if (hw > 0.0) h2 += hw * hw;
            }
            acc += w * w * h2;
        }
    }
    D[t] = acc;
}

// z = r / (D + lambda) per column (z = r where D + lambda is 0)
__global__ void ridge_precond(const float* __restrict__ r, const double* __restrict__ D,
                              const double* __restrict__ lam, int64_t n, int ncol, float* __restrict__ z) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * ncol) return;
    const double m = D[i / ncol] + lam[i % ncol];
    z[i] = m > 0.0 ? (float)((double)r[i] / m) : r[i];
}

constexpr int kDotBlocks = 296;  // fixed grid: deterministic partial order
constexpr int kDotThreads = 256;

// partial[blk][col] = sum over the block's rows of u[row][col] v[row][col]
template <typename U, typename V>
__global__ void __launch_bounds__(kDotThreads) coldot_kernel(const U* u, const V* v, int64_t n,
                                                            int ncol, double* partial) {
    __shared__ double sh[kDotThreads];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nw = kDotThreads / 32;
    for (int c0 = 0; c0 < ncol; c0 += 32) {
        const int c = c0 + lane;
        double acc = 0.0;
        if (c < ncol)
            for (int64_t row = (int64_t)blockIdx.x * nw + warp; row < n;
                 row += (int64_t)gridDim.x * nw)
                acc += (double)u[row * ncol + c] * (double)v[row * ncol + c];
        sh[warp * 32 + lane] = acc;
        __syncthreads();
        if (warp == 0 && c < ncol) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[w * 32 + lane];
            partial[(int64_t)blockIdx.x * ncol + c] = s;
        }
        __syncthreads();
    }
}

__global__ void coldot_reduce(const double* partial, int nblk, int ncol, double* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * ncol + c];
    out[c] = s;
}

// dst[row][c] = src[row][c / rep]
template <typename T>
__global__ void replicate_cols(const T* src, int64_t n, int nsrc, int rep, T* dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int ncol = nsrc * rep;
    if (i >= n * ncol) return;
    const int64_t row = i / ncol;
    const int c = (int)(i - row * ncol);
    dst[i] = src[row * nsrc + c / rep];
}

template <typename A, typename B>
__global__ void convert(const A* a, B* b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (B)a[i];
}

// Ap <- Ap + lambda[c] p
__global__ void add_shift(float* Ap, const float* p, const double* lam, int64_t n, int ncol) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * ncol) return;
    Ap[i] = Ap[i] + (float)lam[i % ncol] * p[i];
}

// x += alpha p; r -= alpha Ap
__global__ void cg_update_xr(float* x, float* r, const float* p, const float* Ap,
                             const double* alpha, int64_t n, int ncol) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * ncol) return;
    const float a = (float)alpha[i % ncol];
    x[i] = x[i] + a * p[i];
    r[i] = r[i] - a * Ap[i];
}

// p = r + beta p
__global__ void cg_update_p(float* p, const float* r, const double* beta, int64_t n, int ncol) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * ncol) return;
    p[i] = r[i] + (float)beta[i % ncol] * p[i];
}

// r = b - (g + lambda x) in FP64; stored in FP64 (for the norm) and FP32
__global__ void refresh_residual(const double* b64, const double* g64, const double* x64,
                                 const double* lam, int64_t n, int ncol, double* r64, float* r) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * ncol) return;
    const double v = b64[i] - (g64[i] + lam[i % ncol] * x64[i]);
    r64[i] = v;
    r[i] = (float)v;
}

// M[i][j] = sum_{k < r} V[i][k] V[j][k] / lam[k]  (V row-major, eigenvectors as columns)
__global__ void tsvd_kernel_matrix(const double* V, const double* lam, int d, int r, double* M) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)d * d) return;
    const int i = (int)(t / d), j = (int)(t - (int64_t)i * d);
    double s = 0.0;
    for (int k = 0; k < r; ++k) s += V[(int64_t)i * d + k] * V[(int64_t)j * d + k] / lam[k];
    M[t] = s;
}

struct DevBuf {
    std::vector<void*> p;
    ~DevBuf() {
        for (void* q : p) cudaFree(q);
    }
    template <typename T>
    bool get(T** out, size_t n) {
        if (cudaMalloc((void**)out, n * sizeof(T) + 16) != cudaSuccess) {
            *out = nullptr;
            return false;
        }
        p.push_back(*out);
        return true;
    }
};

static int nb(int64_t n) { return (int)((n + 255) / 256); }

template <typename U, typename V>
static cudaError_t coldots(const U* u, const V* v, int64_t n, int ncol, double* partial,
                           double* out, cudaStream_t st) {
    coldot_kernel<U, V><<<kDotBlocks, kDotThreads, 0, st>>>(u, v, n, ncol, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    coldot_reduce<<<(ncol + 127) / 128, 128, 0, st>>>(partial, kDotBlocks, ncol, out);
    return cudaGetLastError();
}

#define SOLVE_CUDA(x)                                                            \
    do {                                                                         \
        cudaError_t _e = (x);                                                    \
        if (_e != cudaSuccess) {                                                 \
            set_error("%s: %s (%s:%d)", #x, cudaGetErrorString(_e), __FILE__, __LINE__); \
            return RTT_ECUDA;                                                    \
        }                                                                        \
    } while (0)

}  // namespace rtt

using namespace rtt;

extern "C" rtt_status rtt_solve_ridge(rtt_op op, int arm_mask, const float* data, int n_rhs,
                                      const double* lambdas, int n_lambda, int max_iter,
                                      double tol, int refresh_every, float* x, int* iters_out,
                                      double* relres_out, void* stream) {
    if (!op || !data || !x || !lambdas || n_rhs < 1 || n_lambda < 1 || max_iter < 1 ||
        !(tol > 0.0) || refresh_every < 1 || (int64_t)n_rhs * n_lambda > 65536) {
        set_error("invalid ridge arguments");
        return RTT_EINVAL;
    }
    RTT_TRY(whole_only(op, "the ridge solver"));
    for (int l = 0; l < n_lambda; ++l)
        if (!(lambdas[l] >= 0.0) || !std::isfinite(lambdas[l])) {
            set_error("lambda[%d] = %g must be finite and >= 0", l, lambdas[l]);
            return RTT_EINVAL;
        }
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s != RTT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int ncol = n_rhs * n_lambda;
    const int64_t N = (int64_t)op->n_nodes * op->time.n_hats;
    const int64_t M = (int64_t)seg.total * op->time.n_frames;
    s = ensure_adjoint_scratch(op, ncol, 8);  // the larger of the FP32 and FP64 needs
    if (s == RTT_OK) s = ensure_adjoint_scratch(op, ncol, 4);
    if (s != RTT_OK) return s;
    DevBuf buf;
    float *b1, *r, *p, *Ap, *y, *z;
    double *lam, *partial, *dots, *coef, *x64, *y64, *g64, *b64, *r64, *b1_64, *Dg;
    const int64_t Mm = M > 0 ? M : 1;
    bool ok = buf.get(&b1, N * n_rhs) && buf.get(&r, N * ncol) && buf.get(&p, N * ncol) &&
              buf.get(&z, N * ncol) && buf.get(&Dg, N) &&
              buf.get(&Ap, N * ncol) && buf.get(&y, Mm * ncol) && buf.get(&lam, ncol) &&
              buf.get(&partial, (size_t)kDotBlocks * ncol) && buf.get(&dots, ncol) &&
              buf.get(&coef, 2 * ncol) && buf.get(&x64, N * ncol) && buf.get(&y64, Mm * ncol) &&
              buf.get(&g64, N * ncol) && buf.get(&b64, N * ncol) && buf.get(&r64, N * ncol) &&
              buf.get(&b1_64, N * n_rhs);
    if (!ok) {
        set_error("ridge: device allocation failed (%d columns)", ncol);
        return RTT_ENOMEM;
    }
    std::vector<double> lam_h(ncol), bnorm(ncol), rr(ncol), rr_new(ncol), pap(ncol);
    std::vector<double> alpha(ncol), beta(ncol);
    for (int c = 0; c < ncol; ++c) lam_h[c] = lambdas[c % n_lambda];
    SOLVE_CUDA(cudaMemcpyAsync(lam, lam_h.data(), ncol * 8, cudaMemcpyHostToDevice, st));
    // right-hand side A^T d in FP64 (exact transpose of the FP64 forward)
    convert<float, double><<<nb(M * n_rhs), 256, 0, st>>>(data, y64, M * n_rhs);
    SOLVE_CUDA(cudaGetLastError());
    SOLVE_CUDA(launch_adjoint<double>(op, y64, b1_64, n_rhs, seg, st));
    replicate_cols<double><<<nb(N * ncol), 256, 0, st>>>(b1_64, N, n_rhs, n_lambda, b64);
    SOLVE_CUDA(cudaGetLastError());
    SOLVE_CUDA(coldots(b64, b64, N, ncol, partial, dots, st));
    SOLVE_CUDA(cudaMemcpyAsync(bnorm.data(), dots, ncol * 8, cudaMemcpyDeviceToHost, st));
    // the preconditioner's diagonal (ray level, this arm's rays)
    ridge_diag_kernel<<<nb(N), 256, 0, st>>>(op->cell_ptr, op->c_row, op->c_K0, op->c_F64, op->c_W64, seg,
                                             op->grid.n_r, op->grid.n_phi, op->time.n_hats, op->time.n_frames,
                                             op->delta, Dg);
    SOLVE_CUDA(cudaGetLastError());
    // x = 0, r = b, z = M^-1 r, p = z
    SOLVE_CUDA(cudaMemsetAsync(x, 0, (size_t)N * ncol * 4, st));
    convert<double, float><<<nb(N * ncol), 256, 0, st>>>(b64, r, N * ncol);
    SOLVE_CUDA(cudaGetLastError());
    ridge_precond<<<nb(N * ncol), 256, 0, st>>>(r, Dg, lam, N, ncol, z);
    SOLVE_CUDA(cudaGetLastError());
    SOLVE_CUDA(cudaMemcpyAsync(p, z, (size_t)N * ncol * 4, cudaMemcpyDeviceToDevice, st));
    std::vector<double> rz(ncol), rz_new(ncol);
    SOLVE_CUDA(coldots(r, r, N, ncol, partial, dots, st));
    SOLVE_CUDA(cudaMemcpyAsync(rr.data(), dots, ncol * 8, cudaMemcpyDeviceToHost, st));
    SOLVE_CUDA(coldots(r, z, N, ncol, partial, dots, st));
    SOLVE_CUDA(cudaMemcpyAsync(rz.data(), dots, ncol * 8, cudaMemcpyDeviceToHost, st));
    SOLVE_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < ncol; ++c) bnorm[c] = std::sqrt(bnorm[c]);
    std::vector<char> done(ncol, 0);
    auto converged = [&](int c, double r2) {
        return bnorm[c] == 0.0 || std::sqrt(r2) <= tol * bnorm[c];
    };
    int it = 0;
    bool all_done = true;
    for (int c = 0; c < ncol; ++c) {
        done[c] = converged(c, rr[c]);
        all_done = all_done && done[c];
    }
    while (!all_done && it < max_iter) {
        ++it;
        // Ap = A^T A p + lambda p
        SOLVE_CUDA(launch_forward<float>(op, p, y, ncol, seg, st));
        SOLVE_CUDA(launch_adjoint<float>(op, y, Ap, ncol, seg, st));
        add_shift<<<nb(N * ncol), 256, 0, st>>>(Ap, p, lam, N, ncol);
        SOLVE_CUDA(cudaGetLastError());
        SOLVE_CUDA(coldots(p, Ap, N, ncol, partial, dots, st));
        SOLVE_CUDA(cudaMemcpyAsync(pap.data(), dots, ncol * 8, cudaMemcpyDeviceToHost, st));
        SOLVE_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < ncol; ++c)
            alpha[c] = (done[c] || !(pap[c] > 0.0)) ? 0.0 : rz[c] / pap[c];
        SOLVE_CUDA(cudaMemcpyAsync(coef, alpha.data(), ncol * 8, cudaMemcpyHostToDevice, st));
        cg_update_xr<<<nb(N * ncol), 256, 0, st>>>(x, r, p, Ap, coef, N, ncol);
        SOLVE_CUDA(cudaGetLastError());
        if (it % refresh_every == 0) {
            convert<float, double><<<nb(N * ncol), 256, 0, st>>>(x, x64, N * ncol);
            SOLVE_CUDA(cudaGetLastError());
            SOLVE_CUDA(launch_forward<double>(op, x64, y64, ncol, seg, st));
            SOLVE_CUDA(launch_adjoint<double>(op, y64, g64, ncol, seg, st));
            refresh_residual<<<nb(N * ncol), 256, 0, st>>>(b64, g64, x64, lam, N, ncol, r64, r);
            SOLVE_CUDA(cudaGetLastError());
        }
        ridge_precond<<<nb(N * ncol), 256, 0, st>>>(r, Dg, lam, N, ncol, z);
        SOLVE_CUDA(cudaGetLastError());
        SOLVE_CUDA(coldots(r, r, N, ncol, partial, dots, st));
        SOLVE_CUDA(cudaMemcpyAsync(rr_new.data(), dots, ncol * 8, cudaMemcpyDeviceToHost, st));
        SOLVE_CUDA(coldots(r, z, N, ncol, partial, dots, st));
        SOLVE_CUDA(cudaMemcpyAsync(rz_new.data(), dots, ncol * 8, cudaMemcpyDeviceToHost, st));
        SOLVE_CUDA(cudaStreamSynchronize(st));
        // a column stops only on an FP64 residual: right after a refresh (r
        // was recomputed in FP64 from x), or at the next refresh once the
        // FP32 recurrence says it has converged
        const bool refreshed = it % refresh_every == 0;
        bool want_refresh = false;
        const std::vector<double> rz_prev = rz;
        all_done = true;
        for (int c = 0; c < ncol; ++c) {
            beta[c] = done[c] || rz[c] == 0.0 ? 0.0 : rz_new[c] / rz[c];
            if (!done[c]) {
                rr[c] = rr_new[c];
                rz[c] = rz_new[c];
                if (converged(c, rr[c])) {
                    if (refreshed)
                        done[c] = 1;
                    else
                        want_refresh = true;
                }
            }
            all_done = all_done && done[c];
        }
        if (want_refresh && !all_done) {
            // confirm in FP64 now rather than at the next scheduled refresh
            convert<float, double><<<nb(N * ncol), 256, 0, st>>>(x, x64, N * ncol);
            SOLVE_CUDA(cudaGetLastError());
            SOLVE_CUDA(launch_forward<double>(op, x64, y64, ncol, seg, st));
            SOLVE_CUDA(launch_adjoint<double>(op, y64, g64, ncol, seg, st));
            refresh_residual<<<nb(N * ncol), 256, 0, st>>>(b64, g64, x64, lam, N, ncol, r64, r);
            SOLVE_CUDA(cudaGetLastError());
            ridge_precond<<<nb(N * ncol), 256, 0, st>>>(r, Dg, lam, N, ncol, z);
            SOLVE_CUDA(cudaGetLastError());
            SOLVE_CUDA(coldots(r, r, N, ncol, partial, dots, st));
            SOLVE_CUDA(cudaMemcpyAsync(rr_new.data(), dots, ncol * 8, cudaMemcpyDeviceToHost, st));
            SOLVE_CUDA(coldots(r, z, N, ncol, partial, dots, st));
            SOLVE_CUDA(cudaMemcpyAsync(rz_new.data(), dots, ncol * 8, cudaMemcpyDeviceToHost, st));
            SOLVE_CUDA(cudaStreamSynchronize(st));
            all_done = true;
            for (int c = 0; c < ncol; ++c) {
                if (!done[c]) {
                    // beta from the refreshed residual, as at a scheduled refresh
                    beta[c] = rz_prev[c] == 0.0 ? 0.0 : rz_new[c] / rz_prev[c];
                    rr[c] = rr_new[c];
                    rz[c] = rz_new[c];
                    done[c] = converged(c, rr[c]);
                }
                all_done = all_done && done[c];
            }
        }
        SOLVE_CUDA(cudaMemcpyAsync(coef + ncol, beta.data(), ncol * 8, cudaMemcpyHostToDevice, st));
        cg_update_p<<<nb(N * ncol), 256, 0, st>>>(p, z, coef + ncol, N, ncol);
        SOLVE_CUDA(cudaGetLastError());
    }
    // final FP64 residual ||b - (A^T A + lambda) x|| / ||b|| per column
    convert<float, double><<<nb(N * ncol), 256, 0, st>>>(x, x64, N * ncol);
    SOLVE_CUDA(cudaGetLastError());
    SOLVE_CUDA(launch_forward<double>(op, x64, y64, ncol, seg, st));
    SOLVE_CUDA(launch_adjoint<double>(op, y64, g64, ncol, seg, st));
    refresh_residual<<<nb(N * ncol), 256, 0, st>>>(b64, g64, x64, lam, N, ncol, r64, r);
    SOLVE_CUDA(cudaGetLastError());
    SOLVE_CUDA(coldots(r64, r64, N, ncol, partial, dots, st));
    SOLVE_CUDA(cudaMemcpyAsync(rr_new.data(), dots, ncol * 8, cudaMemcpyDeviceToHost, st));
    SOLVE_CUDA(cudaStreamSynchronize(st));
    bool final_ok = true;
    for (int c = 0; c < ncol; ++c) {
        const double rel = bnorm[c] > 0.0 ? std::sqrt(rr_new[c]) / bnorm[c] : 0.0;
        if (relres_out) relres_out[c] = rel;
        final_ok = final_ok && done[c];
    }
    if (iters_out) *iters_out = it;
    if (!final_ok) {
        set_error("ridge CG: %d iterations without reaching tol %g on every column", it, tol);
        return RTT_ENOTCONVERGED;
    }
    return RTT_OK;
}

extern "C" rtt_status rtt_solve_tsvd(rtt_op op, int arm_mask, const double* Q, int d,
                                     const double* V, const double* evals_host, int rank,
                                     const double* data, int n_rhs, double* xhat, void* stream) {
    if (!op || !Q || !V || !evals_host || !data || !xhat || d < 1 || n_rhs < 1 || rank < 0 ||
        rank > d) {
        set_error("invalid tsvd arguments (d=%d rank=%d n_rhs=%d)", d, rank, n_rhs);
        return RTT_EINVAL;
    }
    RTT_TRY(whole_only(op, "the TSVD solver"));
    for (int k = 0; k < rank; ++k)
        if (!(evals_host[k] > 0.0)) {
            set_error("tsvd: eigenvalue %d = %g is not positive", k, evals_host[k]);
            return RTT_EINVAL;
        }
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s != RTT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = (int64_t)op->n_nodes * op->time.n_hats;
    s = ensure_adjoint_scratch(op, n_rhs, 8);
    if (s != RTT_OK) return s;
    DevBuf buf;
    double *g, *c, *Mx, *coefm, *lam;
    if (!(buf.get(&g, N * n_rhs) && buf.get(&c, (size_t)d * n_rhs) && buf.get(&Mx, (size_t)d * d) &&
          buf.get(&coefm, (size_t)d * n_rhs) && buf.get(&lam, d))) {
        set_error("tsvd: device allocation failed");
        return RTT_ENOMEM;
    }
    SOLVE_CUDA(cudaMemcpyAsync(lam, evals_host, d * 8, cudaMemcpyHostToDevice, st));
    SOLVE_CUDA(launch_adjoint<double>(op, data, g, n_rhs, seg, st));
    tsvd_kernel_matrix<<<nb((int64_t)d * d), 256, 0, st>>>(V, lam, d, rank, Mx);
    SOLVE_CUDA(cudaGetLastError());
    // the three contractions on the tensor cores in FP64 accuracy:
    // c = Q^T g (d x n_rhs), coef = M^T c = M c (M symmetric), xhat = Q coef
    // (as (Q^T)^T coef, with Q^T formed once)
    double* Qt = nullptr;
    if (!buf.get(&Qt, (size_t)d * N)) {
        set_error("tsvd: device allocation failed");
        return RTT_ENOMEM;
    }
    s = gemm_tn_f64(N, d, n_rhs, Q, d, g, n_rhs, c, n_rhs, op->dev_status, st);
    if (s == RTT_OK) s = gemm_tn_f64(d, d, n_rhs, Mx, d, c, n_rhs, coefm, n_rhs, op->dev_status, st);
    if (s == RTT_OK) {
        transpose_kernel<<<dim3((unsigned)((N + 31) / 32), (unsigned)((d + 31) / 32)), dim3(32, 8), 0, st>>>(
            Q, N, d, Qt);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("tsvd: transpose launch failed");
            return RTT_ECUDA;
        }
        s = gemm_tn_f64(d, (int)N, n_rhs, Qt, N, coefm, n_rhs, xhat, n_rhs, op->dev_status, st);
    }
    if (s != RTT_OK) return s;
    SOLVE_CUDA(cudaStreamSynchronize(st));
    return RTT_OK;
}
