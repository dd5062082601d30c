// C = A^T B in FP64 accuracy on the 5th-generation tensor cores, for the
// restricted Gram's contraction (Eq. 21: G = Q^T (A^T A Q)) and the TSVD
// projections.  The method is error-free digit splitting (the Ozaki scheme,
// Ozaki, Ogita, Oishi & Rump 2012, in its integer-digit form):
//
//  * every column c of an operand is scaled by a power of two 2^e_c so its
//    entries lie in (-1, 1), then split exactly into 7 signed digits of 7
//    bits, x 2^-e_c = sum_{s<7} q_s 2^-7(s+1) + r, |q_0| <= 128,
//    |q_{s>=1}| <= 64, |r| <= 2^-50 (q_s = round(128 t), t <- 128 t - q_s);
//    every digit is an integer, exact in BF16;
//  * C_ij = 2^(e_i+f_j) sum_{s,t} 2^-7(s+t+2) sum_k q^A_s[k,i] q^B_t[k,j]:
//    the digit products are integers of at most 14 bits, so a BF16 tensor-
//    core product with FP32 accumulation is exact as long as a sum stays
//    below 2^24: the pairs of one level L = s + t (at most 7 pairs) are
//    accumulated over windows of 128 k in one FP32 TMEM accumulator per
//    level (|sum| < 2^21.7);
//  * after each window the 7 level sums (exact integers) are read out of
//    TMEM and added into two 64-bit integer accumulators per output,
//    hi = sum_{L<=3} v_L 2^7(3-L) and lo = sum_{4<=L<=6} v_L 2^7(6-L) (no
//    overflow for k < 2^27), so the whole reduction, across windows and
//    across the K-split CTAs (integer atomics), is exact and independent of
//    order: the result is deterministic.  Levels L >= 7 (below 2^-49 of
//    2^(e_i+f_j) per product) and the digit remainders are dropped.
//
// tcgen05 pipeline per CTA (one 128 x 64 output tile, one K range): a TMA
// producer warp streams 32-wide K chunks of the 7 A and 7 B digit slices
// (BF16, K-major, 64-byte swizzle) through two shared-memory stages; one
// thread issues tcgen05.mma (M = 128, N = 64, K = 16) for the 28 digit pairs
// into the 7 level accumulators (448 TMEM columns) and commits to mbarriers;
// eight epilogue warps drain TMEM every window.  Every wait is bounded.
#include <cuda_bf16.h>

#include <climits>
#include <vector>

#include "kern_common.cuh"

namespace rtt {

constexpr int kOzDigits = 7;
constexpr int kOzMT = 128;      // output rows per CTA (TMEM lanes)
constexpr int kOzNT = 64;       // output columns per CTA
constexpr int kOzKC = 32;       // K elements per stage (64 bytes of BF16: one swizzle atom)
constexpr int kOzWindow = 128;  // K elements per exact FP32 accumulation window
constexpr int kOzStages = 2;
constexpr int kOzEpiWarps = 8;
constexpr int kOzThreads = (2 + kOzEpiWarps) * 32;
constexpr uint32_t kOzATile = kOzMT * kOzKC * 2;  // 8 KB
constexpr uint32_t kOzBTile = kOzNT * kOzKC * 2;  // 4 KB
constexpr uint32_t kOzStageBytes = kOzDigits * (kOzATile + kOzBTile);  // 84 KB
constexpr int kOzTmemCols = 512;  // 7 levels x 64 columns = 448, allocated as 512

// ---- column exponents: expo[c] = max over rows of frexp's exponent of X[r][c]
__global__ void oz_colmax(int64_t rows, int cols, const double* __restrict__ X, int64_t ldx,
                          int* expo) {
    const int c = blockIdx.y * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    int e = INT_MIN;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const double v = X[r * ldx + c];
        if (v != 0.0) {
            int ex;
            frexp(v, &ex);
            e = max(e, ex);
        }
    }
    if (e != INT_MIN) atomicMax(expo + c, e);
}

// ---- digit slices, transposed to K-major: S[s][c][k] = q_s of X[k][c] 2^-e_c
// (zero in the padding: c >= cols or k >= rows)
__global__ void __launch_bounds__(256) oz_split(int64_t rows, int cols, const double* __restrict__ X,
                                                int64_t ldx, const int* __restrict__ expo,
                                                int cols_pad, int64_t k_pad, __nv_bfloat16* S) {
    __shared__ float tile[kOzDigits][32][33];
    const int64_t k0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int j = ty; j < 32; j += 8) {
        const int64_t k = k0 + j;
        const int c = c0 + tx;
        float q[kOzDigits];
#pragma unroll
        for (int s = 0; s < kOzDigits; ++s) q[s] = 0.0f;
        if (k < rows && c < cols) {
            const int e = expo[c];
            double a = X[k * ldx + c];
            if (e != INT_MIN && a != 0.0) {
                a = ldexp(a, -e);  // exact: |a| < 1
#pragma unroll
                for (int s = 0; s < kOzDigits; ++s) {
                    const double t = a * 128.0;  // exact
                    const double d = rint(t);    // |d| <= 128, then <= 64
                    a = t - d;                   // exact, |a| <= 1/2
                    q[s] = (float)d;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < kOzDigits; ++s) tile[s][j][tx] = q[s];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int c = c0 + j;
        const int64_t k = k0 + tx;
        if (c < cols_pad && k < k_pad) {
#pragma unroll
            for (int s = 0; s < kOzDigits; ++s)
                S[((int64_t)s * cols_pad + c) * k_pad + k] = __float2bfloat16_rn(tile[s][tx][j]);
        }
    }
}

// ---- final scaling: C[i][j] = 2^(e_i + f_j) (hi 2^-35 + lo 2^-56)
__global__ void oz_finish(int m, int n, const long long* __restrict__ acc, const int* __restrict__ ea,
                          const int* __restrict__ eb, int n_pad, double* C, int64_t ldc) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * n) return;
    const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
    double v = 0.0;
    if (ea[i] != INT_MIN && eb[j] != INT_MIN) {
        const long long hi = acc[((int64_t)i * n_pad + j) * 2];
        const long long lo = acc[((int64_t)i * n_pad + j) * 2 + 1];
        const int e = ea[i] + eb[j];
        v = ldexp((double)hi, e - 35) + ldexp((double)lo, e - 56);
    }
    C[(int64_t)i * ldc + j] = v;
}

// ---- the tensor-core kernel ------------------------------------------------

// shared-memory matrix descriptor of a K-major BF16 tile with 64-byte rows
// under the 64-byte swizzle (8-row atoms of 512 bytes)
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused: one atom in K)
    d |= (uint64_t)((512 >> 4) & 0x3FFF) << 32;       // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)4 << 61;                           // 64-byte swizzle
    return d;
}

// instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = 64
constexpr uint32_t kOzIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kOzNT >> 3) << 17) |
                              ((uint32_t)(kOzMT >> 4) << 24);

__device__ __forceinline__ void oz_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(kOzIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void oz_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// exact integer value of an FP32 that holds an integer of magnitude below 2^22
__device__ __forceinline__ int oz_int(float v) {
    return __float_as_int(v + 12582912.0f) - 0x4B400000;
}

struct OzArgs {
    int m_pad, n_pad;
    int64_t k_pad;
    int64_t k_per_cta;  // multiple of kOzWindow
    long long* acc;     // [m_pad][n_pad][2]
    int* status;
};

__global__ void __launch_bounds__(kOzThreads, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
               const OzArgs a) {
    extern __shared__ unsigned char oz_smem_raw[];
    const uint32_t raw = smem_u32(oz_smem_raw);
    const uint32_t base = (raw + 1023) & ~1023u;
    const uint32_t bar_full = base + kOzStages * kOzStageBytes;  // [stages]
    const uint32_t bar_empty = bar_full + 8 * kOzStages;         // [stages]
    const uint32_t bar_tfull = bar_empty + 8 * kOzStages;
    const uint32_t bar_tempty = bar_tfull + 8;
    const uint32_t bar_final = bar_tempty + 8;
    const uint32_t tmem_slot = bar_final + 8;
    unsigned char* slot_ptr = oz_smem_raw + (tmem_slot - raw);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(oz_smem_raw + (tmem_slot + 8 - raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x, nt = blockIdx.y;
    const int64_t k_begin = (int64_t)blockIdx.z * a.k_per_cta;
    int64_t k_end = k_begin + a.k_per_cta;
    if (k_end > a.k_pad) k_end = a.k_pad;
    const int n_chunks = k_end > k_begin ? (int)((k_end - k_begin) / kOzKC) : 0;
    constexpr int kChunksPerWindow = kOzWindow / kOzKC;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kOzStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_full + 8 * s) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_empty + 8 * s) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_tfull) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_tempty), "r"(kOzEpiWarps)
                     : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_final) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 1) {  // TMEM allocation (whole warp)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot),
                     "r"(kOzTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(slot_ptr);

    if (warp == 0) {
        // ---- TMA producer
        if (lane == 0) {
            const uint64_t am = reinterpret_cast<uint64_t>(&amap), bm = reinterpret_cast<uint64_t>(&bmap);
            for (int c = 0; c < n_chunks; ++c) {
                const int st = c % kOzStages;
                const uint32_t ph = (uint32_t)((c / kOzStages) & 1);
                if (c >= kOzStages && !mbar_wait(bar_empty + 8 * st, ph ^ 1)) {
                    *abort_flag = 1;
                    atomicOr(a.status, 1);
                    break;
                }
                if (*abort_flag) break;
                const uint32_t sb = base + st * kOzStageBytes;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_full + 8 * st),
                             "r"(kOzStageBytes)
                             : "memory");
                const int kx = (int)(k_begin + (int64_t)c * kOzKC);
                for (int s = 0; s < kOzDigits; ++s) {
                    const int ra = s * a.m_pad + mt * kOzMT;
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3}], [%4];" ::"r"(sb + s * kOzATile),
                        "l"(am), "r"(kx), "r"(ra), "r"(bar_full + 8 * st)
                        : "memory");
                    const int rb = s * a.n_pad + nt * kOzNT;
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%2, %3}], [%4];" ::"r"(sb + kOzDigits * kOzATile + s * kOzBTile),
                        "l"(bm), "r"(kx), "r"(rb), "r"(bar_full + 8 * st)
                        : "memory");
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            for (int c = 0; c < n_chunks; ++c) {
                const int st = c % kOzStages;
                const uint32_t ph = (uint32_t)((c / kOzStages) & 1);
                const int w = c / kChunksPerWindow, cw = c - w * kChunksPerWindow;
                if (cw == 0 && w > 0 && !mbar_wait(bar_tempty, (uint32_t)((w - 1) & 1))) {
                    *abort_flag = 1;
                    atomicOr(a.status, 1);
                    break;
                }
                if (!mbar_wait(bar_full + 8 * st, ph)) {
                    *abort_flag = 1;
                    atomicOr(a.status, 1);
                    break;
                }
                if (*abort_flag) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sb = base + st * kOzStageBytes;
#pragma unroll 1
                for (int s = 0; s < kOzDigits; ++s) {
                    const uint32_t sa = sb + s * kOzATile;
#pragma unroll 1
                    for (int t = 0; s + t < kOzDigits; ++t) {
                        const uint32_t sbb = sb + kOzDigits * kOzATile + t * kOzBTile;
                        const uint32_t d = tmem + (uint32_t)((s + t) * kOzNT);
#pragma unroll
                        for (int kk = 0; kk < kOzKC / 16; ++kk) {
                            // the first product into a level in a window overwrites it
                            const uint32_t accum = (cw == 0 && kk == 0 && s == 0) ? 0u : 1u;
                            oz_mma(d, oz_desc(sa + 32 * kk), oz_desc(sbb + 32 * kk), accum);
                        }
                    }
                }
                oz_commit(bar_empty + 8 * st);  // the stage is free once these MMAs complete
                if (cw == kChunksPerWindow - 1) oz_commit(bar_tfull);
            }
            // every MMA issued has completed before the TMEM is released
            oz_commit(bar_final);
            if (!mbar_wait(bar_final, 0)) atomicOr(a.status, 1);
        }
    } else {
        // ---- epilogue: rows 32 (warp % 4) + lane, columns 32 h ... 32 h + 31
        const int q = warp & 3, h = (warp - 2) >> 2;
        long long hi[32], lo[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0;
        const int n_windows = n_chunks / kChunksPerWindow;
        bool ok = true;
        for (int w = 0; w < n_windows && ok; ++w) {
            if (!mbar_wait(bar_tfull, (uint32_t)(w & 1))) {
                ok = false;
                if (lane == 0) atomicOr(a.status, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int L = 0; L < kOzDigits; ++L) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(L * kOzNT + 32 * h);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                    "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                      "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
                      "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                      "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
                      "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // level L weighs 2^-7(L+2): hi holds L <= 3 at 2^7(3-L), lo holds L >= 4 at 2^7(6-L)
                const long long sc = L <= 3 ? (1ll << (7 * (3 - L))) : (1ll << (7 * (6 - L)));
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const long long iv = (long long)oz_int(__uint_as_float(v[j])) * sc;
                    if (L <= 3)
                        hi[j] += iv;
                    else
                        lo[j] += iv;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar_tempty) : "memory");
        }
        if (ok && n_windows > 0) {
            const int i = mt * kOzMT + 32 * q + lane;
            unsigned long long* out = reinterpret_cast<unsigned long long*>(a.acc) +
                                      ((int64_t)i * a.n_pad + nt * kOzNT + 32 * h) * 2;
#pragma unroll
            for (int j = 0; j < 32; ++j) {  // integer sums: order-independent
                atomicAdd(out + 2 * j, (unsigned long long)hi[j]);
                atomicAdd(out + 2 * j + 1, (unsigned long long)lo[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols)
                     : "memory");
    }
}

// ---- host ---------------------------------------------------------------------
static int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// C (m x n, row stride ldc) = A^T B with A: k x m (row stride lda), B: k x n
// (row stride ldb), all FP64 device memory.  Workspace is allocated here.
rtt_status gemm_tn_f64(int64_t k, int m, int n, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int* status, cudaStream_t st) {
    if (k < 1 || m < 1 || n < 1 || !A || !B || !C || k >= ((int64_t)1 << 27)) {
        set_error("gemm: invalid arguments (k=%lld m=%d n=%d)", (long long)k, m, n);
        return RTT_EINVAL;
    }
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) {
        set_error("gemm: tensor-map encoder unavailable");
        return RTT_ECUDA;
    }
    const int m_pad = (int)round_up(m, kOzMT), n_pad = (int)round_up(n, kOzNT);
    const int64_t k_pad = round_up(k, kOzWindow);
    const int tiles = (m_pad / kOzMT) * (n_pad / kOzNT);
    const int sms = sm_count();
    int splits = (sms + tiles - 1) / tiles;
    const int64_t windows = k_pad / kOzWindow;
    if (splits > windows) splits = (int)windows;
    const int64_t k_per = round_up((k_pad + splits - 1) / splits, kOzWindow);
    splits = (int)((k_pad + k_per - 1) / k_per);
    __nv_bfloat16 *sa = nullptr, *sb = nullptr;
    int* ex = nullptr;
    long long* acc = nullptr;
    const size_t bytes_a = (size_t)kOzDigits * m_pad * k_pad * 2, bytes_b = (size_t)kOzDigits * n_pad * k_pad * 2;
    cudaError_t e = cudaMalloc(&sa, bytes_a);
    if (e == cudaSuccess) e = cudaMalloc(&sb, bytes_b);
    if (e == cudaSuccess) e = cudaMalloc(&ex, (size_t)(m + n) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&acc, (size_t)m_pad * n_pad * 16);
    auto done = [&](rtt_status s) {
        cudaFree(sa);
        cudaFree(sb);
        cudaFree(ex);
        cudaFree(acc);
        return s;
    };
    if (e != cudaSuccess) {
        set_error("gemm: workspace allocation failed");
        return done(RTT_ENOMEM);
    }
    std::vector<int> init(m + n, INT_MIN);
    cudaMemcpyAsync(ex, init.data(), (size_t)(m + n) * 4, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(acc, 0, (size_t)m_pad * n_pad * 16, st);
    {
        const int gx = (int)(k < 512 ? k : 512);
        oz_colmax<<<dim3(gx, (m + 127) / 128), 128, 0, st>>>(k, m, A, lda, ex);
        oz_colmax<<<dim3(gx, (n + 127) / 128), 128, 0, st>>>(k, n, B, ldb, ex + m);
        oz_split<<<dim3((unsigned)(k_pad / 32), m_pad / 32), 256, 0, st>>>(k, m, A, lda, ex, m_pad, k_pad, sa);
        oz_split<<<dim3((unsigned)(k_pad / 32), n_pad / 32), 256, 0, st>>>(k, n, B, ldb, ex + m, n_pad, k_pad, sb);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            set_error("gemm: split kernels: %s", cudaGetErrorString(e));
            return done(RTT_ECUDA);
        }
    }
    CUtensorMap am, bm;
    {
        cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)kOzDigits * m_pad};
        cuuint64_t strides[1] = {(cuuint64_t)k_pad * 2};
        cuuint32_t box[2] = {kOzKC, kOzMT};
        cuuint32_t es[2] = {1, 1};
        if (enc(&am, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, sa, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            set_error("gemm: tensor map (A) rejected");
            return done(RTT_ECUDA);
        }
        cuuint64_t dimsb[2] = {(cuuint64_t)k_pad, (cuuint64_t)kOzDigits * n_pad};
        cuuint32_t boxb[2] = {kOzKC, kOzNT};
        if (enc(&bm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, sb, dimsb, strides, boxb, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            set_error("gemm: tensor map (B) rejected");
            return done(RTT_ECUDA);
        }
    }
    OzArgs oa;
    oa.m_pad = m_pad;
    oa.n_pad = n_pad;
    oa.k_pad = k_pad;
    oa.k_per_cta = k_per;
    oa.acc = acc;
    oa.status = status;
    const size_t smem = 1024 + (size_t)kOzStages * kOzStageBytes + 8 * (2 * kOzStages + 3) + 16;
    e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        oz_gemm_kernel<<<dim3(m_pad / kOzMT, n_pad / kOzNT, splits), kOzThreads, smem, st>>>(am, bm, oa);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        oz_finish<<<(unsigned)(((int64_t)m * n + 255) / 256), 256, 0, st>>>(m, n, acc, ex, ex + m, n_pad, C, ldc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // before the workspace is freed
    if (e != cudaSuccess) {
        set_error("gemm: %s", cudaGetErrorString(e));
        return done(RTT_ECUDA);
    }
    return done(RTT_OK);
}

}  // namespace rtt

using namespace rtt;

extern "C" rtt_status rtt_gemm_tn_f64(int64_t k, int m, int n, const double* A_dev, int64_t lda,
                                      const double* B_dev, int64_t ldb, double* C_dev, int64_t ldc,
                                      void* stream) {
    if (k < 1 || m < 1 || n < 1 || !A_dev || !B_dev || !C_dev || lda < m || ldb < n || ldc < n ||
        k >= ((int64_t)1 << 27)) {
        set_error("gemm: invalid arguments (k=%lld m=%d n=%d, strides %lld %lld %lld)", (long long)k, m,
                  n, (long long)lda, (long long)ldb, (long long)ldc);
        return RTT_EINVAL;
    }
    int* status = nullptr;
    if (cudaMalloc(&status, 4) != cudaSuccess) {
        set_error("gemm: allocation failed");
        return RTT_ENOMEM;
    }
    cudaMemsetAsync(status, 0, 4, (cudaStream_t)stream);
    rtt_status s = gemm_tn_f64(k, m, n, A_dev, lda, B_dev, ldb, C_dev, ldc, status, (cudaStream_t)stream);
    int hs = 0;
    if (s == RTT_OK) cudaMemcpy(&hs, status, 4, cudaMemcpyDeviceToHost);
    cudaFree(status);
    if (s == RTT_OK && hs) {
        set_error("gemm: a bounded wait of the tensor-core kernel timed out");
        return RTT_ETIMEOUT;
    }
    return s;
}
