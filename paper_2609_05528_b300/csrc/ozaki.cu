// C = A^T B in FP64 accuracy on the 5th-generation tensor cores, for the
// restricted Gram's contraction (Eq. 21: G = Q^T (A^T A Q)) and the TSVD
// projections.  The method is error-free digit splitting (the Ozaki scheme,
// Ozaki, Ogita, Oishi & Rump 2012, in its integer-digit form):
//
//  * every column c of an operand is scaled by a power of two 2^e_c so its
//    entries lie in (-1, 1), rounded to 49 fractional bits and split exactly
//    into 7 signed digits of 7 bits, x 2^-e_c = sum_{s<7} q_s 2^-7(s+1) + r,
//    |q_0| <= 128, q_{s>=1} in [-64, 63] (balanced base 128), |r| <= 2^-50;
//    every digit is an integer, exact in BF16;
//  * C_ij = 2^(e_i+f_j) sum_{s,t} 2^-7(s+t+2) sum_k q^A_s[k,i] q^B_t[k,j]:
//    the digit products are integers of at most 14 bits, so a BF16 tensor-
//    core product with FP32 accumulation is exact as long as a sum stays
//    below 2^24: the pairs of one level L = s + t (at most 7 pairs, at most
//    two of them with the 8-bit leading digit) are accumulated over windows
//    of 256 k in one FP32 TMEM accumulator per level (per k at most
//    2 * 128 * 64 + 5 * 64 * 64 = 36864, so |sum| <= 256 * 36864 < 2^23.2);
//  * after each window the 7 level sums (exact integers) are read out of
//    TMEM and added into two 64-bit integer accumulators per output,
//    hi = sum_{L<=3} v_L 2^7(3-L) and lo = sum_{4<=L<=6} v_L 2^7(6-L) (no
//    overflow for k < 2^27), so the whole reduction, across windows and
//    across the K-split CTAs (integer atomics), is exact and independent of
//    order: the result is deterministic.  Levels L >= 7 (below 2^-49 of
//    2^(e_i+f_j) per product) and the digit remainders are dropped.
//
// tcgen05 pipeline: a persistent CTA per SM walks work units (one 128 x 64
// output tile and one K range each; the K split is chosen so the units fill
// the SMs evenly).  A TMA producer warp streams 32-wide K chunks of the 7 A
// and 7 B digit slices (BF16, K-major, 64-byte swizzle) through two shared-
// memory stages; one thread issues tcgen05.mma (M = 128, N = 64, K = 16) for
// the 28 digit pairs into the 7 level accumulators (448 TMEM columns) and
// commits to mbarriers; sixteen epilogue warps (16 columns each) drain TMEM
// every window.  Every wait is bounded.
#include <cuda_bf16.h>

#include <climits>
#include <mutex>
#include <vector>

#include "kern_common.cuh"

namespace rtt {

constexpr int kOzDigits = 7;
constexpr int kOzMT = 128;      // output rows per CTA (TMEM lanes)
constexpr int kOzNT = 64;       // output columns per CTA
constexpr int kOzKC = 32;       // K elements per stage (64 bytes of BF16: one swizzle atom)
constexpr int kOzWindow = 256;  // K elements per exact FP32 accumulation window
constexpr int kOzStages = 2;
constexpr int kOzEpiWarps = 16;
constexpr int kOzEpiCols = kOzNT * 4 / kOzEpiWarps;  // output columns per epilogue thread (16)
constexpr int kOzThreads = (2 + kOzEpiWarps) * 32;
constexpr uint32_t kOzATile = kOzMT * kOzKC * 2;  // 8 KB
constexpr uint32_t kOzBTile = kOzNT * kOzKC * 2;  // 4 KB
constexpr uint32_t kOzStageBytes = kOzDigits * (kOzATile + kOzBTile);  // 84 KB
constexpr int kOzTmemCols = 512;  // 7 levels x 64 columns = 448, allocated as 512

// ---- column exponents: expo[c] = max over rows of frexp's exponent of X[r][c]
// (read from the exponent field; subnormal entries through frexp)
__device__ __forceinline__ int oz_frexp_exponent(double v) {
    const long long b = __double_as_longlong(v);
    const int field = (int)((b >> 52) & 0x7FF);
    if (field != 0) return field - 1022;
    int ex;
    frexp(v, &ex);
    return ex;
}

__global__ void oz_colmax(int64_t rows, int cols, const double* __restrict__ X, int64_t ldx,
                          int* expo) {
    const int c = blockIdx.y * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    int e = INT_MIN;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const double v = X[r * ldx + c];
        if (v != 0.0) e = max(e, oz_frexp_exponent(v));
    }
    if (e != INT_MIN) atomicMax(expo + c, e);
}

// ---- packed digit slices.  The operand's columns form tiles of R (128 for
// A, 64 for B); for tile t and K chunk ch (32 k) the 7 digit slices are one
// contiguous block of 7 x R rows of 64 bytes, exactly the shared-memory image
// the MMA descriptors read: slice s at s R 64 bytes, row r at r 64 bytes,
// its 16-byte piece j (k = 8 j ... 8 j + 7) at position j ^ ((r >> 1) & 3)
// (the 64-byte swizzle of 512-byte aligned 8-row atoms).  A stage is then two
// contiguous bulk copies.
__host__ __device__ __forceinline__ int64_t oz_packed_index(int s, int c, int64_t k, int R,
                                                            int64_t n_chunks) {
    const int t = c / R, r = c - t * R;
    const int64_t ch = k >> 5;
    const int kk = (int)(k & 31), j = kk >> 3, e = kk & 7;
    const int64_t block = ((int64_t)t * n_chunks + ch) * kOzDigits + s;  // in units of R rows
    return (block * R + r) * 32 + ((j ^ ((r >> 1) & 3)) << 3) + e;     // BF16 elements
}

// q_s of X[k][c] 2^-e_c into the packed slices (zero in the padding:
// c >= cols or k >= rows)
__global__ void __launch_bounds__(256) oz_split(int64_t rows, int cols, const double* __restrict__ X,
                                                int64_t ldx, const int* __restrict__ expo,
                                                int cols_pad, int64_t k_pad, int R, __nv_bfloat16* S) {
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
            const double a = X[k * ldx + c];
            if (e != INT_MIN && a != 0.0) {
                // N = a 2^(49 - e) rounded to the nearest integer (|a 2^-e| < 1,
                // so |N| <= 2^49; the part dropped is at most 2^-50 of 2^e),
                // then its balanced base-128 digits: q_6 ... q_1 in [-64, 63],
                // q_0 = what remains, |q_0| <= 128; all integer arithmetic
                long long N = __double2ll_rn(ldexp(a, 49 - e));
#pragma unroll
                for (int s = kOzDigits - 1; s >= 1; --s) {
                    const long long d = ((N + 64) & 127) - 64;
                    q[s] = (float)d;
                    N = (N - d) >> 7;  // exact: N - d is a multiple of 128
                }
                q[0] = (float)N;
            }
        }
#pragma unroll
        for (int s = 0; s < kOzDigits; ++s) tile[s][j][tx] = q[s];
    }
    __syncthreads();
    const int64_t n_chunks = k_pad >> 5;
    for (int j = ty; j < 32; j += 8) {
        const int c = c0 + j;
        const int64_t k = k0 + tx;
        if (c < cols_pad && k < k_pad) {
#pragma unroll
            for (int s = 0; s < kOzDigits; ++s)
                S[oz_packed_index(s, c, k, R, n_chunks)] = __float2bfloat16_rn(tile[s][tx][j]);
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

// exact integer value of an FP32 that holds an integer (|v| < 2^24)
__device__ __forceinline__ int oz_int(float v) { return __float2int_rn(v); }

struct OzArgs {
    const __nv_bfloat16* sa;  // packed A slices
    const __nv_bfloat16* sb;  // packed B slices
    int m_pad, n_pad;
    int64_t k_pad;
    int64_t k_per_unit;  // multiple of kOzWindow
    int m_tiles, splits;
    int units;           // m_tiles * (n_pad / kOzNT) * splits
    long long* acc;      // [m_pad][n_pad][2]
    int* status;
};

// tile and K range of work unit u (tiles fastest, so concurrent CTAs share
// K ranges of the digit slices in L2)
struct OzUnit {
    int mt, nt;
    int64_t k_begin;
    int n_chunks;
};

__device__ __forceinline__ OzUnit oz_unit(const OzArgs& a, int u) {
    const int tiles = a.m_tiles * (a.n_pad / kOzNT);
    const int tile = u % tiles, sp = u / tiles;
    OzUnit r;
    r.mt = tile % a.m_tiles;
    r.nt = tile / a.m_tiles;
    r.k_begin = (int64_t)sp * a.k_per_unit;
    int64_t k_end = r.k_begin + a.k_per_unit;
    if (k_end > a.k_pad) k_end = a.k_pad;
    r.n_chunks = k_end > r.k_begin ? (int)((k_end - r.k_begin) / kOzKC) : 0;
    return r;
}

__global__ void __launch_bounds__(kOzThreads, 1) oz_gemm_kernel(const OzArgs a) {
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
        // ---- TMA producer: the chunks of this CTA's units, one ring of stages
        if (lane == 0) {
            const int64_t n_chunks_k = a.k_pad / kOzKC;
            int c = 0;  // chunks issued by this CTA
            for (int u = blockIdx.x; u < a.units && !*abort_flag; u += gridDim.x) {
                const OzUnit un = oz_unit(a, u);
                for (int cu = 0; cu < un.n_chunks; ++cu, ++c) {
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
                    const int64_t ch = un.k_begin / kOzKC + cu;
                    const __nv_bfloat16* ga = a.sa + (((int64_t)un.mt * n_chunks_k + ch) * kOzDigits) * kOzMT * kOzKC;
                    const __nv_bfloat16* gb = a.sb + (((int64_t)un.nt * n_chunks_k + ch) * kOzDigits) * kOzNT * kOzKC;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                        ::"r"(sb), "l"(ga), "r"(kOzDigits * kOzATile), "r"(bar_full + 8 * st)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                        ::"r"(sb + kOzDigits * kOzATile), "l"(gb), "r"(kOzDigits * kOzBTile),
                        "r"(bar_full + 8 * st)
                        : "memory");
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            int c = 0, gw = 0;  // chunks and windows consumed by this CTA
            bool live = true;
            for (int u = blockIdx.x; u < a.units && live; u += gridDim.x) {
                const OzUnit un = oz_unit(a, u);
                for (int cu = 0; cu < un.n_chunks; ++cu, ++c) {
                    const int st = c % kOzStages;
                    const uint32_t ph = (uint32_t)((c / kOzStages) & 1);
                    const int cw = cu % kChunksPerWindow;
                    // a new window overwrites the level accumulators: wait
                    // until the epilogue has read the previous window
                    if (cw == 0 && gw > 0 && !mbar_wait(bar_tempty, (uint32_t)((gw - 1) & 1))) {
                        *abort_flag = 1;
                        atomicOr(a.status, 1);
                        live = false;
                        break;
                    }
                    if (!mbar_wait(bar_full + 8 * st, ph)) {
                        *abort_flag = 1;
                        atomicOr(a.status, 1);
                        live = false;
                        break;
                    }
                    if (*abort_flag) {
                        live = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sb = base + st * kOzStageBytes;
                    // descriptors of the stage's first A and B rows; every
                    // operand of the chunk is a constant byte offset from them
                    // (the address field counts 16-byte units)
                    const uint64_t da0 = oz_desc(sb), db0 = oz_desc(sb + kOzDigits * kOzATile);
                    const uint32_t first = cw == 0 ? 0u : 1u;
#pragma unroll
                    for (int s = 0; s < kOzDigits; ++s) {
#pragma unroll
                        for (int t = 0; s + t < kOzDigits; ++t) {
                            const uint32_t d = tmem + (uint32_t)((s + t) * kOzNT);
#pragma unroll
                            for (int kk = 0; kk < kOzKC / 16; ++kk) {
                                // the first product into a level in a window overwrites it
                                const uint32_t accum = (kk == 0 && s == 0) ? first : 1u;
                                oz_mma(d, da0 + (uint64_t)((s * kOzATile + 32 * kk) >> 4),
                                       db0 + (uint64_t)((t * kOzBTile + 32 * kk) >> 4), accum);
                            }
                        }
                    }
                    oz_commit(bar_empty + 8 * st);  // the stage is free once these MMAs complete
                    if (cw == kChunksPerWindow - 1) {
                        oz_commit(bar_tfull);
                        ++gw;
                    }
                }
            }
            // every MMA issued has completed before the TMEM is released
            oz_commit(bar_final);
            if (!mbar_wait(bar_final, 0)) atomicOr(a.status, 1);
        }
    } else {
        // ---- epilogue: rows 32 (warp % 4) + lane, columns kOzEpiCols g ... of
        // the 64 (g = (warp - 2) / 4; a warp reads the TMEM lanes of its
        // quadrant warp % 4)
        const int q = warp & 3, g = (warp - 2) >> 2;
        int gw = 0;  // windows drained by this CTA
        bool ok = true;
        for (int u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
            const OzUnit un = oz_unit(a, u);
            const int n_windows = un.n_chunks / kChunksPerWindow;
            long long hi[kOzEpiCols], lo[kOzEpiCols];
#pragma unroll
            for (int j = 0; j < kOzEpiCols; ++j) hi[j] = lo[j] = 0;
            for (int w = 0; w < n_windows; ++w, ++gw) {
                if (!mbar_wait(bar_tfull, (uint32_t)(gw & 1))) {
                    ok = false;
                    if (lane == 0) atomicOr(a.status, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
                for (int L = 0; L < kOzDigits; ++L) {
                    uint32_t v[kOzEpiCols];
                    const uint32_t taddr =
                        tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(L * kOzNT + kOzEpiCols * g);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                          "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                          "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    // level L weighs 2^-7(L+2): hi holds L <= 3 at 2^7(3-L), lo
                    // holds L >= 4 at 2^7(6-L)
                    const int sh = L <= 3 ? 7 * (3 - L) : 7 * (6 - L);
#pragma unroll
                    for (int j = 0; j < kOzEpiCols; ++j) {
                        const long long iv = (long long)oz_int(__uint_as_float(v[j])) << sh;
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
                const int i = un.mt * kOzMT + 32 * q + lane;
                unsigned long long* out = reinterpret_cast<unsigned long long*>(a.acc) +
                                          ((int64_t)i * a.n_pad + un.nt * kOzNT + kOzEpiCols * g) * 2;
#pragma unroll
                for (int j = 0; j < kOzEpiCols; ++j) {  // integer sums: order-independent
                    atomicAdd(out + 2 * j, (unsigned long long)hi[j]);
                    atomicAdd(out + 2 * j + 1, (unsigned long long)lo[j]);
                }
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

// grow-only workspace per device (kept for the life of the process)
struct OzWorkspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};
constexpr int kOzMaxDevices = 64;
static OzWorkspace g_oz_ws[kOzMaxDevices];
static std::mutex g_oz_ws_mu[kOzMaxDevices];

// C (m x n, row stride ldc) = A^T B with A: k x m (row stride lda), B: k x n
// (row stride ldb), all FP64 device memory.  Workspace is allocated here.
rtt_status gemm_tn_f64(int64_t k, int m, int n, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int* status, cudaStream_t st) {
    if (k < 1 || m < 1 || n < 1 || !A || !B || !C || k >= ((int64_t)1 << 27)) {
        set_error("gemm: invalid arguments (k=%lld m=%d n=%d)", (long long)k, m, n);
        return RTT_EINVAL;
    }
    const int m_pad = (int)round_up(m, kOzMT), n_pad = (int)round_up(n, kOzNT);
    const int64_t k_pad = round_up(k, kOzWindow);
    const int tiles = (m_pad / kOzMT) * (n_pad / kOzNT);
    const int sms = sm_count();
    // K split: the number of units (tiles x splits, whole windows each) whose
    // rounds over the persistent CTAs waste the least, the smallest such
    // count once the waste is below 4%
    const int64_t windows = k_pad / kOzWindow;
    int splits = 1;
    double best = -1.0;
    for (int sp = 1; sp <= 64 && sp <= windows; ++sp) {
        const int64_t per = (windows + sp - 1) / sp;          // windows per unit
        const int64_t used = (windows + per - 1) / per;       // splits actually needed
        const int64_t units = (int64_t)tiles * used;
        const int64_t grid = units < sms ? units : sms;
        const int64_t rounds = (units + grid - 1) / grid;
        // work of the busiest CTA against the even share
        const double eff = (double)windows * tiles / ((double)rounds * per * grid) *
                           ((double)grid / sms);
        if (eff > best + 1e-9) {
            best = eff;
            splits = (int)used;
        }
        if (best >= 0.96) break;
    }
    const int64_t k_per = ((windows + splits - 1) / splits) * kOzWindow;
    splits = (int)((k_pad + k_per - 1) / k_per);
    const int units = tiles * splits;
    const int grid = units < sms ? units : sms;
    // the workspace: digit slices of A and B, column exponents, integer
    // accumulators, from one grow-only per-device buffer held while the call
    // runs (the call synchronises its stream before it returns)
    const size_t bytes_a = (size_t)kOzDigits * m_pad * k_pad * 2, bytes_b = (size_t)kOzDigits * n_pad * k_pad * 2;
    const size_t off_b = (bytes_a + 255) / 256 * 256, off_x = off_b + (bytes_b + 255) / 256 * 256;
    const size_t off_acc = off_x + ((size_t)(m + n) * 4 + 255) / 256 * 256;
    const size_t total = off_acc + (size_t)m_pad * n_pad * 16;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kOzMaxDevices) {
        set_error("gemm: device %d beyond the workspace table", dev);
        return RTT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_oz_ws_mu[dev]);
    OzWorkspace& ws = g_oz_ws[dev];
    cudaError_t e = cudaSuccess;
    if (ws.bytes < total) {
        cudaFree(ws.ptr);
        ws.ptr = nullptr;
        ws.bytes = 0;
        e = cudaMalloc(&ws.ptr, total);
        if (e != cudaSuccess) {
            ws.ptr = nullptr;
            set_error("gemm: workspace allocation of %zu bytes failed", total);
            return RTT_ENOMEM;
        }
        ws.bytes = total;
    }
    unsigned char* base = static_cast<unsigned char*>(ws.ptr);
    __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(base);
    __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(base + off_b);
    int* ex = reinterpret_cast<int*>(base + off_x);
    long long* acc = reinterpret_cast<long long*>(base + off_acc);
    auto done = [&](rtt_status s) { return s; };
    std::vector<int> init(m + n, INT_MIN);
    cudaMemcpyAsync(ex, init.data(), (size_t)(m + n) * 4, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(acc, 0, (size_t)m_pad * n_pad * 16, st);
    {
        const int gx = (int)(k < 512 ? k : 512);
        oz_colmax<<<dim3(gx, (m + 127) / 128), 128, 0, st>>>(k, m, A, lda, ex);
        oz_colmax<<<dim3(gx, (n + 127) / 128), 128, 0, st>>>(k, n, B, ldb, ex + m);
        oz_split<<<dim3((unsigned)(k_pad / 32), m_pad / 32), 256, 0, st>>>(k, m, A, lda, ex, m_pad, k_pad,
                                                                          kOzMT, sa);
        oz_split<<<dim3((unsigned)(k_pad / 32), n_pad / 32), 256, 0, st>>>(k, n, B, ldb, ex + m, n_pad, k_pad,
                                                                          kOzNT, sb);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            set_error("gemm: split kernels: %s", cudaGetErrorString(e));
            return done(RTT_ECUDA);
        }
    }
    OzArgs oa;
    oa.sa = sa;
    oa.sb = sb;
    oa.m_pad = m_pad;
    oa.n_pad = n_pad;
    oa.k_pad = k_pad;
    oa.k_per_unit = k_per;
    oa.m_tiles = m_pad / kOzMT;
    oa.splits = splits;
    oa.units = units;
    oa.acc = acc;
    oa.status = status;
    const size_t smem = 1024 + (size_t)kOzStages * kOzStageBytes + 8 * (2 * kOzStages + 3) + 16;
    e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        oz_gemm_kernel<<<grid, kOzThreads, smem, st>>>(oa);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        oz_finish<<<(unsigned)(((int64_t)m * n + 255) / 256), 256, 0, st>>>(m, n, acc, ex, ex + m, n_pad, C, ldc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // before the workspace is reused
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
