// Adaptive randomized range finder for the restricted normal operator
// H = Q^T A^T A Q of a representation class (Sec. 7-8: the spectra of the
// large classes; Eq. 31 for the operational rank), with an FP64 projected
// eigensolve.  Per block of b caller-supplied Gaussian vectors Omega_i:
//
//   Y = H Omega_i                      (FP64 applies of A and A^T on b columns,
//                                       the contractions with Q on the tensor
//                                       cores in FP64 accuracy)
//   Y <- Y - V (V^T Y), twice           (against the basis found so far)
//   V_i = orthonormal columns of Y by Householder QR with column pivoting
//         (FP64 on the host: the block is at most d x 256), the columns
//         whose pivot falls below 1e-12 of the block's largest column norm
//         before the projection dropped (a factorisation that does not square
//         Y's conditioning: the directions near rho^2 are 1e-8 of the largest);
//         then projected against V again (twice) and factored once more,
//         keeping the columns that keep half their length (a column whose
//         pivot was near the tolerance carries the projection's rounding)
//   W_i = H V_i                         (the operator on the new basis vectors)
//   T = [V_1..V_i]^T [W_1..W_i], symmetrised; its eigenvalues (Jacobi, FP64)
//       are the Ritz values of H on the found subspace
//
// Blocks stop when a block adds no Ritz value at or above rho^2, when the
// basis has all d directions, or after max_blocks.  The Ritz values never
// exceed the eigenvalues of H (Cauchy interlacing), so the rank read from
// them never exceeds the operational rank; once the basis spans the class,
// they are its eigenvalues.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "kern_common.cuh"

extern "C" rtt_status rtt_eig_sym(int n, double* A, double* evals_host, double* V, int max_sweeps,
                                  int* sweeps_host, void* stream);

namespace rtt {

rtt_status gemm_tn_f64(int64_t k, int m, int n, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int* status, cudaStream_t st);

// out[c][r] = in[r][c] for rows x cols (ld_in), out with leading dimension ld_out
__global__ void rf_transpose(const double* __restrict__ in, int64_t rows, int cols, int64_t ld_in,
                             double* __restrict__ out, int64_t ld_out) {
    __shared__ double t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int64_t r = r0 + j;
        const int c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[j][threadIdx.x] = in[r * ld_in + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int c = c0 + j;
        const int64_t r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(int64_t)c * ld_out + r] = t[threadIdx.x][j];
    }
}

// dst[r][c] = src[r][c] (rows x cols, leading dimensions ld_src, ld_dst); sign -1 subtracts
__global__ void rf_copy(const double* __restrict__ src, int64_t ld_src, double* __restrict__ dst,
                        int64_t ld_dst, int64_t rows, int cols, int subtract) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int64_t r = i / cols;
    const int c = (int)(i - r * cols);
    const double v = src[r * ld_src + c];
    if (subtract)
        dst[r * ld_dst + c] -= v;
    else
        dst[r * ld_dst + c] = v;
}

// T <- (T + T^T) / 2 (n x n)
__global__ void rf_symmetrise(double* T, int n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n) return;
    const int r = (int)(i / n), c = (int)(i - (int64_t)r * n);
    if (c <= r) return;
    const double v = 0.5 * (T[(int64_t)r * n + c] + T[(int64_t)c * n + r]);
    T[(int64_t)r * n + c] = v;
    T[(int64_t)c * n + r] = v;
}

static int nb1(int64_t n) { return (int)((n + 255) / 256); }

namespace {
struct Bufs {
    std::vector<void*> p;
    ~Bufs() {
        for (void* q : p) cudaFree(q);
    }
    bool get(double** out, size_t n) {
        if (cudaMalloc(out, (n > 0 ? n : 1) * sizeof(double)) != cudaSuccess) {
            *out = nullptr;
            return false;
        }
        p.push_back(*out);
        return true;
    }
};
}  // namespace

#define RF_TRY(x)                                 \
    do {                                          \
        const rtt_status _s = (x);                \
        if (_s != RTT_OK) return _s;              \
    } while (0)
#define RF_CUDA(x)                                                             \
    do {                                                                       \
        const cudaError_t _e = (x);                                            \
        if (_e != cudaSuccess) {                                               \
            set_error("range finder: %s (%s)", #x, cudaGetErrorString(_e));    \
            return RTT_ECUDA;                                                  \
        }                                                                      \
    } while (0)

struct RfCtx {
    rtt_op_s* op;
    ArmSeg seg;
    const double* Q;  // [N][d]
    double* Qt;       // [d][N]
    int64_t N, M;     // coefficients, arm data samples
    int d;
    double *x, *y, *z;  // apply scratch, c columns
    int c;
    int* status;
    cudaStream_t st;
};

// OUT[:, 0:nc] (d x nc, leading dimension ld_out) = H IN (IN: d x nc, ld_in), in
// sub-blocks of ctx.c columns; sub (d x c) is contiguous scratch
static rtt_status apply_H(RfCtx& cx, const double* IN, int64_t ld_in, double* OUT, int64_t ld_out, int nc,
                          double* sub_in, double* sub_out) {
    for (int j = 0; j < nc; j += cx.c) {
        const int cc = std::min(cx.c, nc - j);
        RF_CUDA((rf_copy<<<nb1((int64_t)cx.d * cc), 256, 0, cx.st>>>(IN + j, ld_in, sub_in, cc, cx.d, cc, 0),
                 cudaGetLastError()));
        // x = Q sub_in (N x cc): C = A^T B with A = Q^T (d x N)
        RF_TRY(gemm_tn_f64(cx.d, (int)cx.N, cc, cx.Qt, cx.N, sub_in, cc, cx.x, cc, cx.status, cx.st));
        RF_TRY(ensure_adjoint_scratch(cx.op, cc, 8));
        RF_CUDA(launch_forward<double>(cx.op, cx.x, cx.y, cc, cx.seg, cx.st));
        RF_CUDA(launch_adjoint<double>(cx.op, cx.y, cx.z, cc, cx.seg, cx.st));
        // sub_out = Q^T z (d x cc)
        RF_TRY(gemm_tn_f64(cx.N, cx.d, cc, cx.Q, cx.d, cx.z, cc, sub_out, cc, cx.status, cx.st));
        RF_CUDA((rf_copy<<<nb1((int64_t)cx.d * cc), 256, 0, cx.st>>>(sub_out, cc, OUT + j, ld_out, cx.d, cc, 0),
                 cudaGetLastError()));
    }
    return RTT_OK;
}

// Householder QR with column pivoting of A (d x b, column-major, host FP64):
// Q (d x r, row-major, leading dimension ldq) spanning the columns whose
// pivot |R_kk| exceeds tol; returns r
static int qr_pivoted(std::vector<double>& A, int d, int b, double tol, double* Q, int ldq) {
    const int kmax = std::min(d, b);
    std::vector<double> norm2(b), beta(kmax);
    std::vector<int> perm(b);
    for (int j = 0; j < b; ++j) {
        perm[j] = j;
        double s = 0.0;
        for (int i = 0; i < d; ++i) s += A[(size_t)j * d + i] * A[(size_t)j * d + i];
        norm2[j] = s;
    }
    int r = 0;
    for (int k = 0; k < kmax; ++k) {
        int p = k;
        for (int j = k + 1; j < b; ++j)
            if (norm2[j] > norm2[p]) p = j;
        if (p != k) {
            for (int i = 0; i < d; ++i) std::swap(A[(size_t)k * d + i], A[(size_t)p * d + i]);
            std::swap(norm2[k], norm2[p]);
            std::swap(perm[k], perm[p]);
        }
        double* a = &A[(size_t)k * d];
        double s = 0.0;
        for (int i = k; i < d; ++i) s += a[i] * a[i];
        const double nrm = std::sqrt(s);
        if (!(nrm > tol)) break;  // the remaining columns are below the tolerance
        const double alpha = a[k] >= 0.0 ? -nrm : nrm;
        // v = a[k:] - alpha e_1, stored in a[k:]; beta = 2 / v^T v
        a[k] -= alpha;
        const double vtv = s - 2.0 * alpha * (a[k] + alpha) + alpha * alpha;  // |a - alpha e1|^2
        beta[k] = vtv > 0.0 ? 2.0 / vtv : 0.0;
        for (int j = k + 1; j < b; ++j) {
            double* c = &A[(size_t)j * d];
            double t = 0.0;
            for (int i = k; i < d; ++i) t += a[i] * c[i];
            t *= beta[k];
            for (int i = k; i < d; ++i) c[i] -= t * a[i];
            // the column's norm below row k (recomputed: no cancellation)
            double q = 0.0;
            for (int i = k + 1; i < d; ++i) q += c[i] * c[i];
            norm2[j] = q;
        }
        r = k + 1;
    }
    // Q = H_0 ... H_{r-1} [I_r; 0]
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < r; ++j) Q[(size_t)i * ldq + j] = i == j ? 1.0 : 0.0;
    std::vector<double> col(d);
    for (int k = r - 1; k >= 0; --k) {
        const double* v = &A[(size_t)k * d];
        for (int j = k; j < r; ++j) {
            double t = 0.0;
            for (int i = k; i < d; ++i) t += v[i] * Q[(size_t)i * ldq + j];
            t *= beta[k];
            for (int i = k; i < d; ++i) Q[(size_t)i * ldq + j] -= t * v[i];
        }
    }
    return r;
}

}  // namespace rtt

using namespace rtt;

extern "C" rtt_status rtt_range_finder(rtt_op op, int arm_mask, const double* Q_dev, int d, int block,
                                       int max_blocks, const double* omega_host, double rho,
                                       double* sigma_out, int* n_sigma_out, int* rank_out,
                                       int* blocks_out, void* stream) {
    if (!op || !Q_dev || d < 1 || d > 4096 || block < 1 || block > 512 || max_blocks < 1 ||
        !omega_host || !(rho > 0.0) || !sigma_out || !n_sigma_out || !rank_out) {
        set_error("invalid range-finder arguments (d=%d block=%d max_blocks=%d)", d, block, max_blocks);
        return RTT_EINVAL;
    }
    RTT_TRY(whole_only(op, "the range finder"));
    ArmSeg seg;
    RTT_TRY(make_seg(op, arm_mask, &seg));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = (int64_t)op->n_nodes * op->time.n_hats;
    const int64_t M = (int64_t)seg.total * op->time.n_frames;
    const int kmax = d;  // the basis never exceeds the class
    const int c = 32;    // apply columns per sub-block
    Bufs bf;
    double *Qt, *x, *y, *z, *V, *HV, *Yb, *tmp, *C, *Vt, *T, *TU, *sub_in, *sub_out;
    int* status = nullptr;
    const int b = block;
    if (!bf.get(&Qt, (size_t)d * N) || !bf.get(&x, (size_t)N * c) || !bf.get(&y, (size_t)(M > 0 ? M : 1) * c) ||
        !bf.get(&z, (size_t)N * c) || !bf.get(&V, (size_t)d * kmax) || !bf.get(&HV, (size_t)d * kmax) ||
        !bf.get(&Yb, (size_t)d * b) || !bf.get(&tmp, (size_t)d * b) ||
        !bf.get(&C, (size_t)kmax * b) || !bf.get(&Vt, (size_t)kmax * d) || !bf.get(&T, (size_t)kmax * kmax) ||
        !bf.get(&TU, (size_t)kmax * kmax) || !bf.get(&sub_in, (size_t)d * c) || !bf.get(&sub_out, (size_t)d * c) ||
        cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
        cudaFree(status);
        set_error("range finder: device allocation failed");
        return RTT_ENOMEM;
    }
    bf.p.push_back(status);
    RF_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    {
        dim3 tg((unsigned)((N + 31) / 32), (unsigned)((d + 31) / 32));
        RF_CUDA((rf_transpose<<<tg, dim3(32, 8), 0, st>>>(Q_dev, N, d, d, Qt, N), cudaGetLastError()));
    }
    RfCtx cx{op, seg, Q_dev, Qt, N, M, d, x, y, z, c, status, st};
    int k = 0, blocks = 0, prev_count = -1;
    std::vector<double> ritz;
    std::vector<double> om((size_t)d * b);
    const double thr = rho * rho;
    for (int i = 0; i < max_blocks && k < kmax; ++i) {
        // Omega_i (d x b) and Y = H Omega_i
        for (int r = 0; r < d; ++r)
            for (int q = 0; q < b; ++q) om[(size_t)r * b + q] = omega_host[(size_t)r * ((size_t)b * max_blocks) + (size_t)i * b + q];
        RF_CUDA(cudaMemcpyAsync(tmp, om.data(), sizeof(double) * d * b, cudaMemcpyHostToDevice, st));
        RF_TRY(apply_H(cx, tmp, b, Yb, b, b, sub_in, sub_out));
        ++blocks;
        // the block's scale before projection (its largest column norm)
        std::vector<double> yh((size_t)d * b);
        RF_CUDA(cudaMemcpyAsync(yh.data(), Yb, sizeof(double) * d * b, cudaMemcpyDeviceToHost, st));
        RF_CUDA(cudaStreamSynchronize(st));
        double ymax = 0.0;
        for (int q = 0; q < b; ++q) {
            double s2 = 0.0;
            for (int r = 0; r < d; ++r) s2 += yh[(size_t)r * b + q] * yh[(size_t)r * b + q];
            ymax = std::max(ymax, std::sqrt(s2));
        }
        // against the basis so far, twice: Y -= V (V^T Y)
        for (int pass = 0; pass < 2 && k > 0; ++pass) {
            RF_TRY(gemm_tn_f64(d, k, b, V, kmax, Yb, b, C, b, status, st));          // C = V^T Y (k x b)
            RF_TRY(gemm_tn_f64(k, d, b, Vt, d, C, b, tmp, b, status, st));           // tmp = V C (d x b)
            RF_CUDA((rf_copy<<<nb1((int64_t)d * b), 256, 0, st>>>(tmp, b, Yb, b, d, b, 1), cudaGetLastError()));
        }
        // orthonormal columns: Householder QR with column pivoting (host FP64;
        // a factorisation that does not square the block's conditioning),
        // pivots below 1e-12 of the block's scale dropped
        RF_CUDA(cudaMemcpyAsync(yh.data(), Yb, sizeof(double) * d * b, cudaMemcpyDeviceToHost, st));
        RF_CUDA(cudaStreamSynchronize(st));
        std::vector<double> acm((size_t)d * b), qh((size_t)d * b);
        for (int r = 0; r < d; ++r)
            for (int q = 0; q < b; ++q) acm[(size_t)q * d + r] = yh[(size_t)r * b + q];
        int nk = qr_pivoted(acm, d, b, 1e-12 * ymax, qh.data(), b);
        RF_CUDA(cudaMemcpyAsync(Yb, qh.data(), sizeof(double) * d * b, cudaMemcpyHostToDevice, st));
        if (nk > 0 && k > 0) {
            // a column whose pivot was near the tolerance carries the rounding
            // of the projection, part of it along V: project the orthonormal
            // columns again (twice) and keep, by a second pivoted QR, those
            // that keep at least half their length
            for (int pass = 0; pass < 2; ++pass) {
                RF_TRY(gemm_tn_f64(d, k, nk, V, kmax, Yb, b, C, nk, status, st));
                RF_TRY(gemm_tn_f64(k, d, nk, Vt, d, C, nk, tmp, nk, status, st));
                RF_CUDA((rf_copy<<<nb1((int64_t)d * nk), 256, 0, st>>>(tmp, nk, Yb, b, d, nk, 1),
                         cudaGetLastError()));
            }
            RF_CUDA(cudaMemcpyAsync(yh.data(), Yb, sizeof(double) * d * b, cudaMemcpyDeviceToHost, st));
            RF_CUDA(cudaStreamSynchronize(st));
            for (int r = 0; r < d; ++r)
                for (int q = 0; q < nk; ++q) acm[(size_t)q * d + r] = yh[(size_t)r * b + q];
            nk = qr_pivoted(acm, d, nk, 0.5, qh.data(), b);
            RF_CUDA(cudaMemcpyAsync(Yb, qh.data(), sizeof(double) * d * b, cudaMemcpyHostToDevice, st));
        }
        if (k + nk > kmax) nk = kmax - k;
        if (nk == 0) break;
        // append the new basis vectors to V (d x kmax) and V^T (kmax x d)
        RF_CUDA((rf_copy<<<nb1((int64_t)d * nk), 256, 0, st>>>(Yb, b, V + k, kmax, d, nk, 0), cudaGetLastError()));
        {
            dim3 tg((unsigned)((d + 31) / 32), (unsigned)((nk + 31) / 32));
            RF_CUDA((rf_transpose<<<tg, dim3(32, 8), 0, st>>>(Yb, d, nk, b, Vt + (int64_t)k * d, d),
                     cudaGetLastError()));
        }
        // H on the new vectors, then the Ritz values on the whole basis
        RF_TRY(apply_H(cx, V + k, kmax, HV + k, kmax, nk, sub_in, sub_out));
        k += nk;
        RF_TRY(gemm_tn_f64(d, k, k, V, kmax, HV, kmax, T, k, status, st));  // T = V^T H V
        RF_CUDA((rf_symmetrise<<<nb1((int64_t)k * k), 256, 0, st>>>(T, k), cudaGetLastError()));
        ritz.assign(k, 0.0);
        RF_TRY(rtt_eig_sym(k, T, ritz.data(), TU, 100, nullptr, stream));
        int count = 0;
        for (double v : ritz) count += v >= thr;
        if (count == prev_count) break;  // the block found nothing new above the threshold
        prev_count = count;
    }
    int st_h = 0;
    RF_CUDA(cudaMemcpyAsync(&st_h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RF_CUDA(cudaStreamSynchronize(st));
    if (st_h) {
        set_error("range finder: a bounded device wait timed out");
        return RTT_ETIMEOUT;
    }
    int rank = 0;
    double margin = 0.0;
    if (k > 0) RF_TRY(rtt_operational_rank(k, ritz.data(), rho, &rank, &margin, sigma_out));
    *n_sigma_out = k;
    *rank_out = rank;
    if (blocks_out) *blocks_out = blocks;
    return RTT_OK;
}
