// Adjoint A^T (Sec. 3.1 Eq. 2-3, the explicit adjoint action of Sec. 5),
// deterministic, without floating-point atomics, by source cells.
//
// A ray e of data row r(e) lies in the source cell (i, j) of its bilinear
// stencil; its four corner weights W_e,c (whitening scale included) feed the
// nodes (i, j), (i+1, j), (i, j+1), (i+1, j+1).  With
//   zhat_e[k][b] = sum_f h_e(f, k) y[r(e)][f][b]
// (h_e the hat weights of the ray's retarded time),
//   x[node][k][b] = sum over the (ray, corner) pairs on that node of
//                   W_e,c zhat_e[k][b].
// The rays are sorted by cell.  A strip i (cells (i, .)) is cut into
// segments of consecutive columns.  One warp takes a (segment, hat group,
// batch chunk) item: for each ray of the segment, in order, it forms
// zhat_e for the group's hats from the ray's staged frames and adds
// W_e,c zhat_e into four register accumulators, for the lower and upper
// node rows of the ray's column and of the next column.  When the walk
// passes a column, that column's two node-row sums are complete for this
// segment and are written as partial records; the last column's successor is
// written at the end.  A gather then forms every node's value as the sum of
// its (at most four) partial records in a fixed order: strip i - 1's upper
// row (segment before, own segment), then strip i's lower row (segment
// before, own segment).  zhat never leaves the SM; the only scratch is the
// partial records (about two to four node rows per cell, read once).
//
// Every output is the same fixed-order sum whatever the launch shape: within
// a record, rays in cell order (then ray order) with fused multiply-adds;
// each zhat in ascending frame order; records in the gather's order.  The
// work items are handed out by an atomic ticket counter (integer, so the
// order in which warps take items changes no bit); the gather resets it.
#include <algorithm>
#include <type_traits>
#include <cub/cub.cuh>
#include <vector>

#include "kern_common.cuh"

namespace rtt {

// segment of a strip: at most this many columns and (unless one column alone
// has more) this many rays.  Longer segments write fewer partial records
// (2 (n + 1) node rows per n columns); 64 and 64 measured best (stress1024
// batch 8: 2.76 -> 2.67 ms, kerr256 0.134 -> 0.120 ms; at 128 the smaller
// workload runs out of items to balance)
constexpr int kSegMaxCols = 64;
constexpr int kSegMaxRays = 64;
// batch columns per pass (records hold one pass)
constexpr int kPassCols32 = 32;
constexpr int kPassCols64 = 16;

struct CellArgs {
    // rays in cell order (cell = the stencil's (i0, j0) node, then ray index)
    const int32_t* c_row;    // input data row
    const int32_t* c_col;    // column j0 of the cell
    const int32_t* c_h0;     // general kernel: hat base K0; TMA kernel: fbase (below)
    const int32_t* c_h1;     // general kernel: 24-bit fraction F0; TMA kernel: phase r0
    const float4* c_W;       // corner weights (whitening scale included)
    const uint2* c_W16;      // their BF16 copy (weights of BF16 precision), or null
    const double* c_W64;     // [4 per ray] the same in FP64
    const double* c_F64;     // exact hat fraction
    const int32_t* seg_ray;  // [n_seg + 1] segment -> positions in the cell order
    const int32_t* seg_col;  // [n_seg] first column
    const int32_t* seg_ncol; // [n_seg] columns
    const int32_t* seg_rec;  // [n_seg] first record (records 2c, 2c + 1: column c, lower / upper)
    ArmSeg seg;
    int seg_rows_all;  // rows of the operator (all orders)
    int K, Tn, B;
    int32_t D;         // 2^24 cadence / hat_step (<= 2^24)
    int b0, Bp;        // this pass: first batch column, columns
    int n_bc;          // batch chunks of the pass
    int n_hg;          // hat groups
    int hw;            // hats per item
    int fwin;          // staged frames per ray (general kernel buffer capacity)
    int64_t n_items;
    int* ctr;          // work ticket counter
    int* status;       // device status word
    const void* y;     // [arm rows][Tn][B]
    void* part;        // [records][K][Bp]
};

// ---------------------------------------------------------------------------
// Work walk shared by both kernels: a warp's sequence of steps.  A RAY step
// is one ray of the current item (in-arm rays only); an END step closes an
// item (its records are written then).  Items come from the ticket counter.
// ---------------------------------------------------------------------------
struct Step {
    int kind;        // 0 done, 1 ray, 2 item end
    int pos;         // ray: position in the cell order
    int row_out;     // ray: output row
    int col;         // ray: column relative to the segment's first column
    int h0, h1;      // ray: hat coordinate (general kernel: K0, F0; TMA kernel: first
                     // frame of the ray's hat-0 taps and its weight phase r0)
    int rec0, ncol;  // item: first record, columns
    int g, bc;       // item: hat group and batch chunk
};

struct Walk {
    int64_t item = -1;
    int pos = 0, end = 0, col0 = 0, ncol = 0, rec0 = 0, g = 0, bc = 0;
    bool open = false;
};

__device__ __forceinline__ int64_t take_ticket(int* ctr, int lane) {
    int t = 0;
    if (lane == 0) t = atomicAdd(ctr, 1);
    return (int64_t)__shfl_sync(0xffffffffu, t, 0);
}

// next step of the warp's walk (warp-uniform); a ray step's fields are plain
// loads at its position, so the kernels fetch them two steps before use
__device__ __forceinline__ Step walk_next(const CellArgs& a, Walk& w, int lane) {
    Step s;
    s.kind = 0;
    const bool all_rows = a.seg.total == a.seg_rows_all;
    if (!w.open) {
        w.item = take_ticket(a.ctr, lane);
        if (w.item >= a.n_items) return s;  // done
        const int64_t q = w.item / a.n_bc;
        w.bc = (int)(w.item - q * a.n_bc);
        const int sg = (int)(q / a.n_hg);
        w.g = (int)(q - (int64_t)sg * a.n_hg);
        w.pos = a.seg_ray[sg];
        w.end = a.seg_ray[sg + 1];
        w.col0 = a.seg_col[sg];
        w.ncol = a.seg_ncol[sg];
        w.rec0 = a.seg_rec[sg];
        w.open = true;
    }
    s.rec0 = w.rec0;
    s.ncol = w.ncol;
    s.g = w.g;
    s.bc = w.bc;
    while (w.pos < w.end) {
        const int p = w.pos++;
        const int row = a.c_row[p];
        const int row_out = all_rows ? row : seg_out_row(a.seg, row);
        if (row_out < 0) continue;  // not in the arm
        s.kind = 1;
        s.pos = p;
        s.row_out = row_out;
        s.col = a.c_col[p] - w.col0;
        s.h0 = a.c_h0[p];
        s.h1 = a.c_h1[p];
        return s;
    }
    w.open = false;
    s.kind = 2;
    return s;
}

// Register accumulators of an item: lower / upper node-row sums of the
// current column (lc, uc) and of the next column (ln, un), NH hats x BC
// columns per lane.  A ray adds its corners (i,j), (i+1,j) to the current
// column and (i,j+1), (i+1,j+1) to the next; passing a column writes the
// current sums and moves the next column's into their place.
template <typename T, int NH, int BC>
struct ColAcc {
    T lc[NH][BC], uc[NH][BC], ln[NH][BC], un[NH][BC];
    __device__ __forceinline__ void zero_all() {
#pragma unroll
        for (int h = 0; h < NH; ++h)
#pragma unroll
            for (int b = 0; b < BC; ++b) lc[h][b] = uc[h][b] = ln[h][b] = un[h][b] = T(0);
    }
    __device__ __forceinline__ void shift() {
#pragma unroll
        for (int h = 0; h < NH; ++h)
#pragma unroll
            for (int b = 0; b < BC; ++b) {
                lc[h][b] = ln[h][b];
                uc[h][b] = un[h][b];
                ln[h][b] = T(0);
                un[h][b] = T(0);
            }
    }
    __device__ __forceinline__ void add(const T (&z)[NH][BC], T w0, T w1, T w2, T w3) {
#pragma unroll
        for (int h = 0; h < NH; ++h)
#pragma unroll
            for (int b = 0; b < BC; ++b) {
                lc[h][b] = fmac(w0, z[h][b], lc[h][b]);
                uc[h][b] = fmac(w1, z[h][b], uc[h][b]);
                ln[h][b] = fmac(w2, z[h][b], ln[h][b]);
                un[h][b] = fmac(w3, z[h][b], un[h][b]);
            }
    }
};

// FP32 with packed pairs (each component rounded as fmac)
template <int NH, int BC>
__device__ __forceinline__ void acc_add2(ColAcc<float, NH, BC>& A, const float (&z)[NH][BC],
                                         float4 w) {
    static_assert(BC % 2 == 0, "pairs");
    const float2 w0 = make_float2(w.x, w.x), w1 = make_float2(w.y, w.y), w2 = make_float2(w.z, w.z),
                 w3 = make_float2(w.w, w.w);
#pragma unroll
    for (int h = 0; h < NH; ++h)
#pragma unroll
        for (int b = 0; b < BC; b += 2) {
            const float2 zz = make_float2(z[h][b], z[h][b + 1]);
            float2 t = __ffma2_rn(w0, zz, make_float2(A.lc[h][b], A.lc[h][b + 1]));
            A.lc[h][b] = t.x;
            A.lc[h][b + 1] = t.y;
            t = __ffma2_rn(w1, zz, make_float2(A.uc[h][b], A.uc[h][b + 1]));
            A.uc[h][b] = t.x;
            A.uc[h][b + 1] = t.y;
            t = __ffma2_rn(w2, zz, make_float2(A.ln[h][b], A.ln[h][b + 1]));
            A.ln[h][b] = t.x;
            A.ln[h][b + 1] = t.y;
            t = __ffma2_rn(w3, zz, make_float2(A.un[h][b], A.un[h][b + 1]));
            A.un[h][b] = t.x;
            A.un[h][b + 1] = t.y;
        }
}

// Where an item writes: record row (rec, hat k) of the pass holds Bp
// columns; the item's batch chunk starts at column boff and has nb of them.
// Lanes at or beyond `nlanes` hold no hat of the item and write nothing.
// A lane whose registers hold its column quads in the order q ^ qx (qx = 0
// or 1: the TMA kernel's bank-spreading order, whose records are always
// whole 16-byte quads) writes register quad q to column quad q ^ qx.
struct EmitAt {
    int kbase, boff, nb, nlanes;
    bool vec;
    int qx = 0;
};

// write one slot's two records (hats k_h = kbase + lane + 32 h)
template <typename T, int NH, int BC>
__device__ __forceinline__ void emit_slot(const CellArgs& a, const T (&lo)[NH][BC],
                                          const T (&up)[NH][BC], int rec, const EmitAt& at,
                                          int lane) {
    if (lane >= at.nlanes) return;
    T* part = reinterpret_cast<T*>(a.part);
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        const int k = at.kbase + lane + 32 * h;
        if (k >= a.K) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            T* o = part + ((int64_t)(rec + half) * a.K + k) * a.Bp + at.boff;
            const T(&v)[BC] = half ? up[h] : lo[h];
            if constexpr (sizeof(T) == 4 && BC % 4 == 0) {
                if (at.vec) {
#pragma unroll
                    for (int q = 0; q < BC / 4; ++q)
                        reinterpret_cast<float4*>(o)[q ^ at.qx] =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    continue;
                }
            }
            if constexpr (sizeof(T) == 8 && BC % 2 == 0) {
                if (at.vec) {
#pragma unroll
                    for (int q = 0; q < BC / 2; ++q)
                        reinterpret_cast<double2*>(o)[q] = make_double2(v[2 * q], v[2 * q + 1]);
                    continue;
                }
            }
#pragma unroll
            for (int b = 0; b < BC; ++b)
                if (b < at.nb) o[b] = v[b];
        }
    }
}

// pass the current column: write its records, move the next column's sums in
template <typename T, int NH, int BC>
__device__ __forceinline__ void next_column(const CellArgs& a, ColAcc<T, NH, BC>& A, int rec,
                                            const EmitAt& at, int lane) {
    emit_slot(a, A.lc, A.uc, rec, at, lane);
    A.shift();
}

// close an item: write every column not yet written and the successor column
template <typename T, int NH, int BC>
__device__ __forceinline__ void finish_item(const CellArgs& a, ColAcc<T, NH, BC>& A, int& jc,
                                            const Step& s, const EmitAt& at, int lane) {
    for (; jc < s.ncol; ++jc) next_column(a, A, s.rec0 + 2 * jc, at, lane);
    emit_slot(a, A.lc, A.uc, s.rec0 + 2 * s.ncol, at, lane);
    A.zero_all();
    jc = 0;
}

// ---------------------------------------------------------------------------
// TMA kernel (FP32, the whole batch in one chunk, B = BC in {4, 8, 16}, a
// periodic cadence of P frames per hat step with F = 32 / BC frames per
// 128-byte line dividing P).  Per ray step the item's frames (HG groups of
// 32 hats: (32 HG + 1) P frames) arrive by one 3D tensor copy of 128-byte
// lines under the 128-byte swizzle, double-buffered over the warp's steps;
// frames before 0 or after the last are zero-filled by the copy.  The
// contraction per hat is one fused multiply-add chain over its 2P taps in
// ascending frame order (the general kernel's order).
// ---------------------------------------------------------------------------
constexpr int kCellWarps = 4;

template <int BC, int P, int HG>
struct CellBox {
    static constexpr int kF = 32 / BC;  // frames per 128-byte line
    static_assert(P % kF == 0, "a line holds a whole number of frames that divides P");
    static constexpr int kRows = ((32 * HG + 1) * P + 2 * (kF - 1)) / kF;
    static constexpr uint32_t kBytes = (uint32_t)kRows * 128;
    static constexpr uint32_t kStride = (kBytes + 1023) & ~1023u;
};

// taps of HG hats of one lane for the frame residue M: lines rs + d.  The
// lane's register quad q holds column quad q ^ qx: at BC = 16 consecutive
// lanes' taps lie two 128-byte lines apart, so under the 128-byte swizzle a
// warp's reads of one quad would meet only four bank groups; with the
// neighbouring quad read by half of the lanes they meet all eight (each
// output's chain of taps is unchanged).
template <int BC, int P, int HG, int M>
__device__ __forceinline__ void cell_contract(const unsigned char* buf, int rs0, int qx,
                                              const float (&wt)[2 * P], float (&z)[HG][BC]) {
    constexpr int Q = BC / 4;
    constexpr int F = 32 / BC;
    constexpr int ND = (M + 2 * P - 1) / F + 1;
#pragma unroll
    for (int h = 0; h < HG; ++h) {
        const int rs = rs0 - h * (32 * P / F);
        uint32_t A[ND], X[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            A[d] = (uint32_t)(rs + d) * 128u;
            X[d] = (uint32_t)((rs + d) & 7) << 4;
        }
#pragma unroll
        for (int b = 0; b < BC; ++b) z[h][b] = 0.0f;
#pragma unroll
        for (int j = 0; j < 2 * P; ++j) {
            const int dj = (M + j) / F, cj = (M + j) % F;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const uint32_t off = A[dj] | ((uint32_t)(16 * (cj * Q + (q ^ qx))) ^ X[dj]);
                const float4 v = *reinterpret_cast<const float4*>(buf + off);
                fmac2x2(wt[j], v, z[h][4 * q + 0], z[h][4 * q + 1], z[h][4 * q + 2], z[h][4 * q + 3]);
            }
        }
    }
}

template <int BC, int P, int HG>
__device__ __forceinline__ void cell_contract_any(int M, const unsigned char* buf, int rs0, int qx,
                                                  const float (&wt)[2 * P], float (&z)[HG][BC]) {
    constexpr int F = 32 / BC;
    if constexpr (F == 1) {
        cell_contract<BC, P, HG, 0>(buf, rs0, qx, wt, z);
    } else if constexpr (F == 2) {
        if (M == 0) cell_contract<BC, P, HG, 0>(buf, rs0, qx, wt, z);
        else cell_contract<BC, P, HG, 1>(buf, rs0, qx, wt, z);
    } else if constexpr (F == 4) {
        switch (M) {
            case 0: cell_contract<BC, P, HG, 0>(buf, rs0, qx, wt, z); break;
            case 1: cell_contract<BC, P, HG, 1>(buf, rs0, qx, wt, z); break;
            case 2: cell_contract<BC, P, HG, 2>(buf, rs0, qx, wt, z); break;
            default: cell_contract<BC, P, HG, 3>(buf, rs0, qx, wt, z); break;
        }
    } else {
        switch (M) {
            case 0: cell_contract<BC, P, HG, 0>(buf, rs0, qx, wt, z); break;
            case 1: cell_contract<BC, P, HG, 1>(buf, rs0, qx, wt, z); break;
            case 2: cell_contract<BC, P, HG, 2>(buf, rs0, qx, wt, z); break;
            case 3: cell_contract<BC, P, HG, 3>(buf, rs0, qx, wt, z); break;
            case 4: cell_contract<BC, P, HG, 4>(buf, rs0, qx, wt, z); break;
            case 5: cell_contract<BC, P, HG, 5>(buf, rs0, qx, wt, z); break;
            case 6: cell_contract<BC, P, HG, 6>(buf, rs0, qx, wt, z); break;
            default: cell_contract<BC, P, HG, 7>(buf, rs0, qx, wt, z); break;
        }
    }
}

// CTAs per SM the TMA kernel's registers are set for: three (the shared
// memory's limit), two at BC = 16, whose four 16-column accumulators do not
// fit in a third of the register file without spilling in the tap loop
template <int BC>
struct CellTmaOcc {
    static constexpr int kMinBlocks = BC == 16 ? 2 : 3;
};

template <int BC, int P, int HG>
__global__ void __launch_bounds__(kCellWarps * 32, CellTmaOcc<BC>::kMinBlocks)
adj_cell_tma_kernel(const __grid_constant__ CUtensorMap ymap, const CellArgs a) {
    static_assert(BC == 4 || BC == 8 || BC == 16, "128-byte lines of whole frames");
    wait_prior_grid();
    constexpr int F = CellBox<BC, P, HG>::kF;
    constexpr int LGF = F == 1 ? 0 : (F == 2 ? 1 : (F == 4 ? 2 : 3));
    constexpr uint32_t BOX_BYTES = CellBox<BC, P, HG>::kBytes;
    constexpr uint32_t BUF_STRIDE = CellBox<BC, P, HG>::kStride;
    constexpr int HATS = 32 * HG;
    extern __shared__ unsigned char smem_cell_raw[];
    const uint32_t raw_u32 = smem_u32(smem_cell_raw);
    const uint32_t base_u32 = (raw_u32 + 1023) & ~1023u;  // swizzle atom alignment
    unsigned char* base = smem_cell_raw + (base_u32 - raw_u32);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned char* bufp0 = base + (size_t)(2 * warp) * BUF_STRIDE;
    const uint32_t buf0 = base_u32 + (2 * warp) * BUF_STRIDE;
    const uint32_t bar0 = base_u32 + kCellWarps * 2 * BUF_STRIDE + 16 * warp;
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int32_t D32 = a.D;
    const uint64_t tmap = reinterpret_cast<uint64_t>(&ymap);
    // copy coordinates of a ray step: first line R4 and the item's frame offset in it
    struct Cp {
        int R4, sbase;
        int32_t r0;
        float4 w;
    };
    auto derive = [&](const Step& s, Cp& c) {
        const int fbase = s.h0;  // first frame of hat 0's taps
        c.r0 = s.h1;             // weight phase: tap j of every hat weighs 1 - |r0 - j D| 2^-24
        const int kg0 = HATS * s.g;
        const int f_lo = fbase - P * (kg0 + HATS - 1);  // first frame of the item's last hat
        c.R4 = f_lo >> LGF;                              // floor division (f_lo may be < 0)
        c.sbase = fbase - P * kg0 - c.R4 * F;            // >= 0
        c.w = corner_weights(a.c_W, a.c_W16, s.pos);
    };
    auto issue = [&](const Step& s, const Cp& c, uint32_t b) {
        if (lane != 0) return;
        const uint32_t bar = bar0 + 8u * b, dst = buf0 + b * BUF_STRIDE;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(BOX_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
            "l"(tmap), "r"(0), "r"(c.R4), "r"(s.row_out), "r"(bar)
            : "memory");
    };
    Walk wk;
    ColAcc<float, HG, BC> A;
    A.zero_all();
    int jc = 0;
    uint32_t n_issued = 0, n_done = 0;  // ray copies issued / consumed
    // steps s0 (consumed now), s1 (copy in flight), s2 (fields loading)
    Step s0 = walk_next(a, wk, lane);
    Step s1 = s0.kind ? walk_next(a, wk, lane) : s0;
    Step s2 = s1.kind ? walk_next(a, wk, lane) : s1;
    Cp c0{}, c1{};
    if (s0.kind == 1) {
        derive(s0, c0);
        issue(s0, c0, n_issued++ & 1);
    }
    if (s1.kind == 1) {
        derive(s1, c1);
        issue(s1, c1, n_issued++ & 1);
    }
    EmitAt at{0, 0, BC, 32, true};
    // register quad q holds column quad q ^ qx: at BC = 16 the swizzle phase of
    // a lane's taps repeats every four lanes, so lanes 4-7 of each eight take
    // the neighbouring quad (eight bank groups per read instead of four)
    const int qx = BC == 16 ? ((lane >> 2) & 1) : 0;
    at.qx = qx;
    while (s0.kind) {
        at.kbase = HATS * s0.g;
        if (s0.kind == 1) {
            const uint32_t b = n_done & 1;
            if (!mbar_wait(bar0 + 8u * b, (n_done >> 1) & 1)) {
                if (lane == 0) atomicOr(a.status, 1);
                if (n_issued > n_done + 1)
                    mbar_wait(bar0 + 8u * ((n_done + 1) & 1), ((n_done + 1) >> 1) & 1);
                return;
            }
            float wt[2 * P];
#pragma unroll
            for (int j = 0; j < 2 * P; ++j)
                wt[j] = 1.0f - (float)abs(c0.r0 - j * D32) * (1.0f / (float)kFracOne);
            const int s0f = c0.sbase - P * lane;
            float z[HG][BC];
            cell_contract_any<BC, P, HG>(s0f & (F - 1), bufp0 + b * BUF_STRIDE, s0f >> LGF, qx, wt, z);
            __syncwarp();  // buffer b is free for the next copy issued into it
            ++n_done;
            for (; jc < s0.col; ++jc) next_column(a, A, s0.rec0 + 2 * jc, at, lane);
            acc_add2(A, z, c0.w);
        } else {
            finish_item(a, A, jc, s0, at, lane);
        }
        s0 = s1;
        c0 = c1;
        s1 = s2;
        s2 = s1.kind ? walk_next(a, wk, lane) : s1;
        if (s1.kind == 1) {
            derive(s1, c1);
            issue(s1, c1, n_issued++ & 1);
        }
    }
}

// ---------------------------------------------------------------------------
// TMA kernel for 32- and 64-column passes (FP32; any batch of whole passes, a
// periodic cadence of P in {2, 4, 8} frames per hat step).  A pass's frame
// record is PW / 32 whole 128-byte lines, so a ray step's frames arrive by
// one tensor copy of the pass's columns (the tensor map's frame stride is
// the batch's) under the 128-byte swizzle, as in adj_cell_tma_kernel.
// PW / 16 lanes share a hat: lane (h, c) = (lane / L, lane % L) holds the
// 16 columns 16 c .. 16 c + 15 of hat h of the item's 32 / L, so its
// accumulators are those of the 16-column kernel.  Its register quad q holds
// column quad q ^ (h & 3) of its 16: consecutive hats' taps lie P frames
// apart, and with the quads spread this way a warp's reads of a quad meet all
// eight bank groups (at P = 2, 4 and 8).  Each output's tap chain, the walk
// and the records are the other kernels' (the same bits).
// ---------------------------------------------------------------------------
template <int PW, int P>
struct CellBoxPass {
    static constexpr int kL = PW / 16;            // lanes per hat
    static constexpr int kW = 32 / kL;            // hats per item
    static constexpr int kG = PW / 32;            // 128-byte lines per frame
    static constexpr int kFrames = (kW + 1) * P;  // frames per ray step
    static constexpr uint32_t kBytes = (uint32_t)kFrames * kG * 128;
    static constexpr uint32_t kStride = (kBytes + 1023) & ~1023u;
};

template <int PW, int P>
__global__ void __launch_bounds__(kCellWarps * 32, 2)
adj_cell_tma_pass_kernel(const __grid_constant__ CUtensorMap ymap, const CellArgs a) {
    static_assert(PW == 32 || PW == 64, "32- or 64-column passes");
    wait_prior_grid();
    using Box = CellBoxPass<PW, P>;
    constexpr int L = Box::kL, W = Box::kW, G = Box::kG;
    constexpr uint32_t BOX_BYTES = Box::kBytes;
    constexpr uint32_t BUF_STRIDE = Box::kStride;
    extern __shared__ unsigned char smem_cellp_raw[];
    const uint32_t raw_u32 = smem_u32(smem_cellp_raw);
    const uint32_t base_u32 = (raw_u32 + 1023) & ~1023u;  // swizzle atom alignment
    unsigned char* base = smem_cellp_raw + (base_u32 - raw_u32);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = lane / L, c = lane % L;  // the lane's hat in the item and its 16 columns
    const int qx = h & 3;                   // register quad q holds column quad q ^ qx of them
    const unsigned char* bufp0 = base + (size_t)(2 * warp) * BUF_STRIDE;
    const uint32_t buf0 = base_u32 + (2 * warp) * BUF_STRIDE;
    const uint32_t bar0 = base_u32 + kCellWarps * 2 * BUF_STRIDE + 16 * warp;
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int32_t D32 = a.D;
    const uint64_t tmap = reinterpret_cast<uint64_t>(&ymap);
    struct Cp {
        int R;  // first frame of the box: the item's last hat's first tap
        int32_t r0;
        float4 w;
    };
    auto derive = [&](const Step& s, Cp& cp) {
        cp.r0 = s.h1;  // weight phase: tap j of every hat weighs 1 - |r0 - j D| 2^-24
        cp.R = s.h0 - P * (W * s.g + W - 1);
        cp.w = corner_weights(a.c_W, a.c_W16, s.pos);
    };
    auto issue = [&](const Step& s, const Cp& cp, uint32_t b) {
        if (lane != 0) return;
        const uint32_t bar = bar0 + 8u * b, dst = buf0 + b * BUF_STRIDE;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(BOX_BYTES)
                     : "memory");
        if constexpr (G == 1) {
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
                "l"(tmap), "r"(0), "r"(cp.R), "r"(s.row_out), "r"(bar)
                : "memory");
        } else {
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
                "l"(tmap), "r"(0), "r"(0), "r"(cp.R), "r"(s.row_out), "r"(bar)
                : "memory");
        }
    };
    // records of the current column: hat kbase + h, columns 16 c .. of the pass
    auto emit = [&](const float (&lo)[1][16], const float (&up)[1][16], int rec, int kbase) {
        const int k = kbase + h;
        if (k >= a.K) return;
        float* part = reinterpret_cast<float*>(a.part);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float4* o = reinterpret_cast<float4*>(part + ((int64_t)(rec + half) * a.K + k) * a.Bp + 16 * c);
            const float(&v)[16] = half ? up[0] : lo[0];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                o[q ^ qx] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
    };
    Walk wk;
    ColAcc<float, 1, 16> A;
    A.zero_all();
    int jc = 0;
    uint32_t n_issued = 0, n_done = 0;  // ray copies issued / consumed
    // steps s0 (consumed now), s1 (copy in flight), s2 (fields loading)
    Step s0 = walk_next(a, wk, lane);
    Step s1 = s0.kind ? walk_next(a, wk, lane) : s0;
    Step s2 = s1.kind ? walk_next(a, wk, lane) : s1;
    Cp c0{}, c1{};
    if (s0.kind == 1) {
        derive(s0, c0);
        issue(s0, c0, n_issued++ & 1);
    }
    if (s1.kind == 1) {
        derive(s1, c1);
        issue(s1, c1, n_issued++ & 1);
    }
    while (s0.kind) {
        const int kbase = W * s0.g;
        if (s0.kind == 1) {
            const uint32_t b = n_done & 1;
            if (!mbar_wait(bar0 + 8u * b, (n_done >> 1) & 1)) {
                if (lane == 0) atomicOr(a.status, 1);
                if (n_issued > n_done + 1)
                    mbar_wait(bar0 + 8u * ((n_done + 1) & 1), ((n_done + 1) >> 1) & 1);
                return;
            }
            float wt[2 * P];
#pragma unroll
            for (int j = 0; j < 2 * P; ++j)
                wt[j] = 1.0f - (float)abs(c0.r0 - j * D32) * (1.0f / (float)kFracOne);
            const unsigned char* buf = bufp0 + b * BUF_STRIDE;
            const int fb0 = P * (W - 1 - h);  // box frame of the lane's first tap
            float z[1][16];
#pragma unroll
            for (int k = 0; k < 16; ++k) z[0][k] = 0.0f;
#pragma unroll
            for (int j = 0; j < 2 * P; ++j) {
                const uint32_t line = (uint32_t)(G * (fb0 + j) + (c >> 1));
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t chunk = (uint32_t)(4 * (c & 1) + (q ^ qx)) ^ (line & 7u);
                    const float4 v = *reinterpret_cast<const float4*>(buf + line * 128u + chunk * 16u);
                    fmac2x2(wt[j], v, z[0][4 * q + 0], z[0][4 * q + 1], z[0][4 * q + 2], z[0][4 * q + 3]);
                }
            }
            __syncwarp();  // buffer b is free for the next copy issued into it
            ++n_done;
            for (; jc < s0.col; ++jc) {
                emit(A.lc, A.uc, s0.rec0 + 2 * jc, kbase);
                A.shift();
            }
            acc_add2(A, z, c0.w);
        } else {
            // close the item: every column not yet written, then the successor column
            for (; jc < s0.ncol; ++jc) {
                emit(A.lc, A.uc, s0.rec0 + 2 * jc, kbase);
                A.shift();
            }
            emit(A.lc, A.uc, s0.rec0 + 2 * s0.ncol, kbase);
            A.zero_all();
            jc = 0;
        }
        s0 = s1;
        c0 = c1;
        s1 = s2;
        s2 = s1.kind ? walk_next(a, wk, lane) : s1;
        if (s1.kind == 1) {
            derive(s1, c1);
            issue(s1, c1, n_issued++ & 1);
        }
    }
}

// ---------------------------------------------------------------------------
// Direct-load kernel for batches of one or two columns (FP32, a periodic
// cadence of P in {2, 4, 8} frames per hat step).  A frame record is 4 or 8
// bytes, too small for the staged kernels' 16-byte pieces, so each lane (a
// hat of the item's 32 HG) reads its 2P taps straight from y through L1
// (neighbouring lanes' windows overlap by half); the taps of the next ray
// step are loaded while the current one is contracted.  Taps outside the
// observation read as zero, as the TMA kernels' out-of-bounds fill.  The
// walk, tap weights, fused multiply-add chains, accumulators and records are
// adj_cell_tma_kernel's: the same bits.
// ---------------------------------------------------------------------------
template <int BC, int P, int HG>
__global__ void __launch_bounds__(kCellWarps * 32, 4)
adj_cell_direct_kernel(const CellArgs a) {
    static_assert(BC == 1 || BC == 2, "one or two columns");
    wait_prior_grid();
    constexpr int HATS = 32 * HG;
    constexpr int NT = 2 * P;  // taps per hat
    const int lane = threadIdx.x & 31;
    const float* y = reinterpret_cast<const float*>(a.y);
    const int32_t D32 = a.D;
    // the taps of a ray step: hat kg0 + lane + 32 h reads frames fbase - P k + j
    auto load_taps = [&](const Step& s, float (&t)[HG][NT][BC]) {
        const float* yr = y + (int64_t)s.row_out * a.Tn * BC;
        const int kg0 = HATS * s.g;
#pragma unroll
        for (int h = 0; h < HG; ++h) {
            const int f0 = s.h0 - P * (kg0 + lane + 32 * h);
            const bool inside = f0 >= 0 && f0 + NT <= a.Tn;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int f = f0 + j;
                const bool ok = inside || (f >= 0 && f < a.Tn);
#pragma unroll
                for (int b = 0; b < BC; ++b) t[h][j][b] = ok ? __ldg(yr + (int64_t)f * BC + b) : 0.0f;
            }
        }
    };
    Walk wk;
    ColAcc<float, HG, BC> A;
    A.zero_all();
    int jc = 0;
    Step s0 = walk_next(a, wk, lane);
    Step s1 = s0.kind ? walk_next(a, wk, lane) : s0;
    float t0[HG][NT][BC], t1[HG][NT][BC];
    if (s0.kind == 1) load_taps(s0, t0);
    EmitAt at{0, 0, BC, 32, false};
    while (s0.kind) {
        if (s1.kind == 1) load_taps(s1, t1);  // the next step's taps, in flight during this one
        at.kbase = HATS * s0.g;
        if (s0.kind == 1) {
            float wt[NT];
#pragma unroll
            for (int j = 0; j < NT; ++j)
                wt[j] = 1.0f - (float)abs(s0.h1 - j * D32) * (1.0f / (float)kFracOne);
            float z[HG][BC];
#pragma unroll
            for (int h = 0; h < HG; ++h)
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    float acc = 0.0f;
#pragma unroll
                    for (int j = 0; j < NT; ++j) acc = __fmaf_rn(wt[j], t0[h][j][b], acc);
                    z[h][b] = acc;
                }
            for (; jc < s0.col; ++jc) next_column(a, A, s0.rec0 + 2 * jc, at, lane);
            const float4 w = corner_weights(a.c_W, a.c_W16, s0.pos);
            A.add(z, w.x, w.y, w.z, w.w);
        } else {
            finish_item(a, A, jc, s0, at, lane);
        }
        s0 = s1;
#pragma unroll
        for (int h = 0; h < HG; ++h)
#pragma unroll
            for (int j = 0; j < NT; ++j)
#pragma unroll
                for (int b = 0; b < BC; ++b) t0[h][j][b] = t1[h][j][b];
        s1 = s0.kind ? walk_next(a, wk, lane) : s0;
    }
}

// ---------------------------------------------------------------------------
// General kernel (FP32 or FP64; any cadence, batch chunk and alignment).  An
// item covers hw <= 32 hats (lane = hat).  Per ray step the frames those hats
// touch are staged by per-lane asynchronous copies into a padded
// shared-memory buffer (16 bytes of padding every 4 frames: lanes whose
// frames lie a hat step apart read different banks), double-buffered over the
// warp's steps.  Hat k sums the frames with (k - 1) 2^24 <= U(f) <
// (k + 1) 2^24 in ascending order: with the 24-bit fixed-point weight
// 1 - |U(f) - k 2^24| 2^-24 in FP32 (the TMA kernel's taps, hence its bits),
// with the exact FP64 fraction in FP64.
// ---------------------------------------------------------------------------
constexpr int kGenWarps = 4;

__host__ __device__ __forceinline__ int stage_off(int fl, int E) { return fl * E + (fl >> 2) * 16; }

template <typename T>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src, int bytes) {
    if (bytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

template <typename T, int BC>
__global__ void __launch_bounds__(kGenWarps * 32)
adj_cell_gen_kernel(const CellArgs a, uint32_t buf_bytes, int vec_stage) {
    wait_prior_grid();
    extern __shared__ __align__(16) unsigned char smem_gen_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* bufp0 = smem_gen_raw + (size_t)(2 * warp) * buf_bytes;
    const uint32_t buf0 = smem_u32(bufp0);
    constexpr int E = BC * (int)sizeof(T);  // staged bytes per frame
    const T* y = reinterpret_cast<const T*>(a.y);
    const int64_t D = a.D;
    struct Cp {
        int fa, nf;  // staged frames [fa, fa + nf)
        int64_t U0;
        double F64;
        T w[4];
    };
    auto derive = [&](const Step& s, Cp& c) {
        c.U0 = (int64_t)s.h0 * kFracOne + (int64_t)s.h1;
        const int kg0 = a.hw * s.g;
        // frames with (kg0 - 1) 2^24 <= U(f) < (kg0 + hw) 2^24
        int64_t fa = floor_div(c.U0 - (int64_t)(kg0 + a.hw) * kFracOne, D) + 1;
        int64_t fb = floor_div(c.U0 - (int64_t)(kg0 - 1) * kFracOne, D);
        if (fa < 0) fa = 0;
        if (fb > a.Tn - 1) fb = a.Tn - 1;
        c.fa = (int)fa;
        c.nf = fb >= fa ? (int)(fb - fa + 1) : 0;  // <= fwin by the choice of hw
        if constexpr (sizeof(T) == 8) {
            c.F64 = a.c_F64[s.pos];
            const double2* p = reinterpret_cast<const double2*>(a.c_W64 + 4 * (int64_t)s.pos);
            const double2 v0 = p[0], v1 = p[1];
            c.w[0] = v0.x; c.w[1] = v0.y; c.w[2] = v1.x; c.w[3] = v1.y;
        } else {
            const float4 v = corner_weights(a.c_W, a.c_W16, s.pos);
            c.w[0] = v.x; c.w[1] = v.y; c.w[2] = v.z; c.w[3] = v.w;
            c.F64 = 0.0;
        }
    };
    auto issue = [&](const Step& s, const Cp& c, uint32_t b) {
        const uint32_t dst = buf0 + b * buf_bytes;
        const int bcol = s.bc * BC;
        const int nb = a.Bp - bcol < BC ? a.Bp - bcol : BC;
        const T* src = y + ((int64_t)s.row_out * a.Tn + c.fa) * a.B + a.b0 + bcol;
        if (vec_stage) {  // 16-byte pieces (E a multiple of 16, aligned rows, whole chunks)
            constexpr int QE = E / 16 > 0 ? E / 16 : 1;
            for (int o = lane; o < c.nf * QE; o += 32) {
                const int fl = o / QE, q = o - fl * QE;
                cp_async<T>(dst + stage_off(fl, E) + 16 * q,
                            reinterpret_cast<const unsigned char*>(src + (int64_t)fl * a.B) + 16 * q, 16);
            }
        } else {
            for (int o = lane; o < c.nf * BC; o += 32) {
                const int fl = o / BC, bb = o - fl * BC;
                if (bb < nb)
                    cp_async<T>(dst + stage_off(fl, E) + bb * (int)sizeof(T), src + (int64_t)fl * a.B + bb,
                                (int)sizeof(T));
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    Walk wk;
    ColAcc<T, 1, BC> A;
    A.zero_all();
    int jc = 0;
    uint32_t n_issued = 0, n_done = 0;
    Step s0 = walk_next(a, wk, lane);
    Step s1 = s0.kind ? walk_next(a, wk, lane) : s0;
    Step s2 = s1.kind ? walk_next(a, wk, lane) : s1;
    Cp c0{}, c1{};
    if (s0.kind == 1) {
        derive(s0, c0);
        issue(s0, c0, n_issued++ & 1);
    }
    if (s1.kind == 1) {
        derive(s1, c1);
        issue(s1, c1, n_issued++ & 1);
    }
    EmitAt at{0, 0, BC, a.hw, false};
    while (s0.kind) {
        at.kbase = a.hw * s0.g;
        at.boff = s0.bc * BC;
        at.nb = a.Bp - at.boff < BC ? a.Bp - at.boff : BC;
        if (s0.kind == 1) {
            // s0's group is complete once at most the one after it is pending
            if (n_issued > n_done + 1)
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            else
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncwarp();
            const unsigned char* buf = bufp0 + (n_done & 1) * buf_bytes;
            T z[1][BC];
#pragma unroll
            for (int b = 0; b < BC; ++b) z[0][b] = T(0);
            const int k = at.kbase + lane;
            if (lane < a.hw && k < a.K) {
                const int64_t hi_excl = (int64_t)(k + 1) * kFracOne;
                const int64_t lo_incl = (int64_t)(k - 1) * kFracOne;
                int64_t f = floor_div(c0.U0 - hi_excl, D) + 1;  // first frame with U(f) < hi
                if (f < c0.fa) f = c0.fa;
                int64_t U = c0.U0 - f * D;
                for (; f < c0.fa + c0.nf && U >= lo_incl; ++f, U -= D) {
                    const int32_t Ur = (int32_t)(U - (int64_t)k * kFracOne);  // [-2^24, 2^24)
                    T hw;
                    if constexpr (sizeof(T) == 4) {
                        hw = 1.0f - (float)abs(Ur) * (1.0f / (float)kFracOne);
                    } else {
                        // exact fraction of u(f) = u0 - f cadence / hat_step, u0 = K0 + F64
                        const double R = (double)((f * D) & kFracMask) * (1.0 / (double)kFracOne);
                        double v = c0.F64 - R;
                        if (v < 0.0) v += 1.0;
                        hw = (Ur >= 0) ? 1.0 - v : v;
                    }
                    const T* vv = reinterpret_cast<const T*>(buf + stage_off((int)(f - c0.fa), E));
#pragma unroll
                    for (int b = 0; b < BC; ++b) z[0][b] = fmac(hw, vv[b], z[0][b]);
                }
            }
            __syncwarp();  // buffer free for the copy issued into it next
            ++n_done;
            for (; jc < s0.col; ++jc) next_column(a, A, s0.rec0 + 2 * jc, at, lane);
            A.add(z, c0.w[0], c0.w[1], c0.w[2], c0.w[3]);
        } else {
            finish_item(a, A, jc, s0, at, lane);
        }
        s0 = s1;
        c0 = c1;
        s1 = s2;
        s2 = s1.kind ? walk_next(a, wk, lane) : s1;
        if (s1.kind == 1) {
            derive(s1, c1);
            issue(s1, c1, n_issued++ & 1);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Periodic staged kernel (FP32 or FP64; a frame step of 1/P hat step, P in
// {2, 4, 8}; any batch, in chunks of BC columns).  An item covers 32 NH hats
// (lane l: hats l + 32 h).  Per ray step the item's (32 NH + 1) P frames of
// the chunk are staged by per-lane asynchronous copies into the padded
// buffer of the general kernel, double-buffered over the warp's steps.  Hat
// k sums its 2P taps, frames fbase - P k + j in ascending order, with the
// TMA kernel's FP32 weights 1 - |r0 - j D| 2^-24 (hence its bits) or, in
// FP64, the exact weights of the ray's FP64 hat fraction (taps j < P carry
// 1 - frac, taps j >= P carry frac).  Frames outside the observation are
// skipped.
// ---------------------------------------------------------------------------
template <typename T, int BC, int P, int NH>
__global__ void __launch_bounds__(kGenWarps * 32, 3)
adj_cell_per_kernel(const CellArgs a, uint32_t buf_bytes, int vec_stage) {
    wait_prior_grid();
    extern __shared__ __align__(16) unsigned char smem_per_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* bufp0 = smem_per_raw + (size_t)(2 * warp) * buf_bytes;
    const uint32_t buf0 = smem_u32(bufp0);
    constexpr int E = BC * (int)sizeof(T);  // staged bytes per frame
    constexpr int HATS = 32 * NH;
    const T* y = reinterpret_cast<const T*>(a.y);
    const int32_t D32 = a.D;
    struct Cp {
        int fa, nf;   // staged frames [fa, fa + nf)
        int fbase;    // first tap frame of hat 0
        int32_t r0;   // FP32 weight phase
        T w[4];
    };
    auto derive = [&](const Step& s, Cp& c) {
        c.fbase = s.h0;
        c.r0 = s.h1;
        const int kg0 = HATS * s.g;
        int fa = c.fbase - P * (kg0 + HATS - 1);
        int fb = c.fbase - P * kg0 + 2 * P - 1;
        if (fa < 0) fa = 0;
        if (fb > a.Tn - 1) fb = a.Tn - 1;
        c.fa = fa;
        c.nf = fb >= fa ? fb - fa + 1 : 0;  // <= (HATS + 1) P = fwin
        if constexpr (sizeof(T) == 8) {
            const double2* p = reinterpret_cast<const double2*>(a.c_W64 + 4 * (int64_t)s.pos);
            const double2 v0 = p[0], v1 = p[1];
            c.w[0] = v0.x; c.w[1] = v0.y; c.w[2] = v1.x; c.w[3] = v1.y;
        } else {
            const float4 v = corner_weights(a.c_W, a.c_W16, s.pos);
            c.w[0] = v.x; c.w[1] = v.y; c.w[2] = v.z; c.w[3] = v.w;
        }
    };
    auto issue = [&](const Step& s, const Cp& c, uint32_t b) {
        const uint32_t dst = buf0 + b * buf_bytes;
        const int bcol = s.bc * BC;
        const int nb = a.Bp - bcol < BC ? a.Bp - bcol : BC;
        const T* src = y + ((int64_t)s.row_out * a.Tn + c.fa) * a.B + a.b0 + bcol;
        if (vec_stage) {
            constexpr int QE = E / 16 > 0 ? E / 16 : 1;
            for (int o = lane; o < c.nf * QE; o += 32) {
                const int fl = o / QE, q = o - fl * QE;
                cp_async<T>(dst + stage_off(fl, E) + 16 * q,
                            reinterpret_cast<const unsigned char*>(src + (int64_t)fl * a.B) + 16 * q, 16);
            }
        } else {
            for (int o = lane; o < c.nf * BC; o += 32) {
                const int fl = o / BC, bb = o - fl * BC;
                if (bb < nb)
                    cp_async<T>(dst + stage_off(fl, E) + bb * (int)sizeof(T), src + (int64_t)fl * a.B + bb,
                                (int)sizeof(T));
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    Walk wk;
    ColAcc<T, NH, BC> A;
    A.zero_all();
    int jc = 0;
    uint32_t n_issued = 0, n_done = 0;
    Step s0 = walk_next(a, wk, lane);
    Step s1 = s0.kind ? walk_next(a, wk, lane) : s0;
    Step s2 = s1.kind ? walk_next(a, wk, lane) : s1;
    Cp c0{}, c1{};
    if (s0.kind == 1) {
        derive(s0, c0);
        issue(s0, c0, n_issued++ & 1);
    }
    if (s1.kind == 1) {
        derive(s1, c1);
        issue(s1, c1, n_issued++ & 1);
    }
    EmitAt at{0, 0, BC, 32, false};
    while (s0.kind) {
        at.kbase = HATS * s0.g;
        at.boff = s0.bc * BC;
        at.nb = a.Bp - at.boff < BC ? a.Bp - at.boff : BC;
        if (s0.kind == 1) {
            if (n_issued > n_done + 1)
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            else
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncwarp();
            const unsigned char* buf = bufp0 + (n_done & 1) * buf_bytes;
            T wt[2 * P];
            if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int j = 0; j < 2 * P; ++j)
                    wt[j] = 1.0f - (float)abs(c0.r0 - j * D32) * (1.0f / (float)kFracOne);
            } else {
                // exact fraction of u(f) at the taps' frames: F64 - (f D mod 2^24) 2^-24, mod 1
                const double F64 = a.c_F64[s0.pos];
#pragma unroll
                for (int j = 0; j < 2 * P; ++j) {
                    const int64_t f = (int64_t)c0.fbase + j;  // any hat: P k D is a whole step
                    const int64_t fd = f * (int64_t)D32;
                    const double R = (double)(((fd % kFracOne) + kFracOne) & kFracMask) *
                                     (1.0 / (double)kFracOne);
                    double v = F64 - R;
                    if (v < 0.0) v += 1.0;
                    wt[j] = j < P ? 1.0 - v : v;
                }
            }
            T z[NH][BC];
#pragma unroll
            for (int h = 0; h < NH; ++h) {
#pragma unroll
                for (int b = 0; b < BC; ++b) z[h][b] = T(0);
                const int k = at.kbase + lane + 32 * h;
                const int f0 = c0.fbase - P * k;  // first tap frame
                if (k < a.K) {
#pragma unroll
                    for (int j = 0; j < 2 * P; ++j) {
                        const int fl = f0 + j - c0.fa;
                        if (fl >= 0 && fl < c0.nf) {
                            const T* vv = reinterpret_cast<const T*>(buf + stage_off(fl, E));
                            if constexpr (sizeof(T) == 4 && BC % 4 == 0) {
#pragma unroll
                                for (int q = 0; q < BC / 4; ++q) {
                                    const float4 v = reinterpret_cast<const float4*>(vv)[q];
                                    fmac2x2(wt[j], v, z[h][4 * q], z[h][4 * q + 1], z[h][4 * q + 2],
                                            z[h][4 * q + 3]);
                                }
                            } else {
#pragma unroll
                                for (int b = 0; b < BC; ++b) z[h][b] = fmac(wt[j], vv[b], z[h][b]);
                            }
                        }
                    }
                }
            }
            __syncwarp();  // buffer free for the copy issued into it next
            ++n_done;
            for (; jc < s0.col; ++jc) next_column(a, A, s0.rec0 + 2 * jc, at, lane);
            if constexpr (sizeof(T) == 4 && BC % 2 == 0)
                acc_add2(A, z, make_float4(c0.w[0], c0.w[1], c0.w[2], c0.w[3]));
            else
                A.add(z, c0.w[0], c0.w[1], c0.w[2], c0.w[3]);
        } else {
            finish_item(a, A, jc, s0, at, lane);
        }
        s0 = s1;
        c0 = c1;
        s1 = s2;
        s2 = s1.kind ? walk_next(a, wk, lane) : s1;
        if (s1.kind == 1) {
            derive(s1, c1);
            issue(s1, c1, n_issued++ & 1);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Gather: x[node][k][b0 + b] = sum of the node's records in the fixed order
// (strip i - 1 upper row: segment before, own; strip i lower row: segment
// before, own).  Also resets the work ticket counter for the next adjoint.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
adj_gather_kernel(const int32_t* gslot, const T* part, T* x, int64_t n_nodes, int K, int B, int b0,
                  int Bp, int* ctr) {
    wait_prior_grid();
    if (blockIdx.x == 0 && threadIdx.x == 0) *ctr = 0;
    const int64_t per_node = (int64_t)K * Bp;
    const int64_t n = n_nodes * per_node;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = i / per_node;
        const int64_t r = i - node * per_node;  // k * Bp + b
        const int k = (int)(r / Bp), b = (int)(r - (int64_t)k * Bp);
        const int4 sl = *reinterpret_cast<const int4*>(gslot + 4 * node);
        T v = T(0);
        bool first = true;
        const int s4[4] = {sl.x, sl.y, sl.z, sl.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (s4[q] >= 0) {
                const T t = part[(int64_t)s4[q] * per_node + r];
                v = first ? t : v + t;
                first = false;
            }
        x[(node * K + k) * B + b0 + b] = v;
    }
}

// 16-byte version (FP32, Bp, B and b0 multiples of 4, aligned buffers)
__global__ void __launch_bounds__(256)
adj_gather4_kernel(const int32_t* gslot, const float* part, float* x, int64_t n_nodes, int K, int B,
                   int b0, int Bp, int* ctr) {
    wait_prior_grid();
    if (blockIdx.x == 0 && threadIdx.x == 0) *ctr = 0;
    const int64_t per_node4 = (int64_t)K * Bp / 4;
    const int64_t n = n_nodes * per_node4;
    const int Bp4 = Bp / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = i / per_node4;
        const int64_t r = i - node * per_node4;
        const int k = (int)(r / Bp4), q = (int)(r - (int64_t)k * Bp4);
        const int4 sl = *reinterpret_cast<const int4*>(gslot + 4 * node);
        const int s4[4] = {sl.x, sl.y, sl.z, sl.w};
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        bool first = true;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (s4[j] >= 0) {
                const float4 t = __ldcs(reinterpret_cast<const float4*>(part) + s4[j] * per_node4 + r);
                if (first) {
                    v = t;
                    first = false;
                } else {
                    v.x += t.x;
                    v.y += t.y;
                    v.z += t.z;
                    v.w += t.w;
                }
            }
        *reinterpret_cast<float4*>(x + (node * K + k) * B + b0 + 4 * q) = v;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// batch columns per pass: 16 in FP64, 32 in FP32 (64 at batches of whole
// 64-column passes, which the TMA pass kernel reads as two lines per frame)
static int pass_cols(int elem, int batch) {
    if (elem == 8) return kPassCols64;
    return batch % 64 == 0 ? 2 * kPassCols32 : kPassCols32;
}

size_t adjoint_scratch_bytes(const rtt_op_s* op, int batch, int elem) {
    const int bp = batch < pass_cols(elem, batch) ? batch : pass_cols(elem, batch);
    return (size_t)op->n_rec * op->time.n_hats * (size_t)bp * (size_t)elem;
}

rtt_status ensure_adjoint_scratch(rtt_op_s* op, int batch, int elem) {
    const size_t bytes = adjoint_scratch_bytes(op, batch, elem);
    if (op->cpart_bytes >= bytes) return RTT_OK;
    if (op->cpart) {
        cudaDeviceSynchronize();
        cudaFree(op->cpart);
        op->cpart = nullptr;
        op->cpart_bytes = 0;
    }
    if (cudaMalloc(&op->cpart, bytes) != cudaSuccess) {
        op->cpart = nullptr;
        set_error("adjoint partial records: allocation of %zu bytes failed", bytes);
        return RTT_ENOMEM;
    }
    op->cpart_bytes = bytes;
    return RTT_OK;
}

// ray tables in cell order
// ray tables in cell order; with a periodic cadence (P frames per hat step,
// D = 2^24 / P) also each ray's first tap frame of hat 0, c0 + 1 - P with
// c0 = floor(U0 / D), and its weight phase r0 = U0 - (c0 + 1) D + 2^24 in
// [2^24 - D, 2^24): hat k's taps are the frames fbase - P k + j, j < 2P, with
// weights 1 - |r0 - j D| 2^-24 (U0 = K0 2^24 + F0, the fixed-point hat
// coordinate of frame 0)
__global__ void cell_tables(int64_t E, int n_phi, int P, int64_t D, const int32_t* cray,
                            const int32_t* ray_row, const int32_t* node00, const int32_t* K0,
                            const int32_t* F0, const float4* W, const double* W64, const double* F64,
                            int32_t* c_row, int32_t* c_col, int32_t* c_K0, int32_t* c_F0,
                            int32_t* c_fb, int32_t* c_r0, float4* c_W, double* c_W64,
                            double* c_F64) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= E) return;
    const int e = cray[p];
    c_row[p] = ray_row[e];
    c_col[p] = node00[e] % n_phi;
    c_K0[p] = K0[e];
    c_F0[p] = F0[e];
    if (P > 0) {
        const int64_t U0 = (int64_t)K0[e] * kFracOne + (int64_t)F0[e];
        const int64_t c0 = floor_div(U0, D);
        c_fb[p] = (int32_t)(c0 + 1 - P);
        c_r0[p] = (int32_t)(U0 - (c0 + 1) * D) + kFracOne;
    }
    c_W[p] = W[e];
    for (int c = 0; c < 4; ++c) c_W64[4 * p + c] = W64[4 * (int64_t)e + c];
    c_F64[p] = F64[e];
}

// Cell structures of a built operator (ray tables in cell order, strip
// segments, record bases, gather table).  The row-ordered ray tables must be
// complete on the device.
rtt_status build_cells(rtt_op_s* op, cudaStream_t st) {
    const int64_t E = op->n_rays;
    const int n_r = op->grid.n_r, n_phi = op->grid.n_phi;
    const int64_t S = op->n_nodes;
    const int n_strips = n_r - 1;
    const int64_t n_cells = (int64_t)n_strips * n_phi;
    // rays sorted by cell (= node00, the stencil's (i0, j0) node), stable in ray index
    int32_t *keys_out = nullptr, *vals_in = nullptr, *cray = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    int end_bit = 1;
    while ((1ll << end_bit) < S) ++end_bit;
    auto cleanup = [&]() {
        cudaFree(keys_out);
        cudaFree(vals_in);
        cudaFree(cray);
        cudaFree(tmp);
        keys_out = vals_in = cray = nullptr;
        tmp = nullptr;
    };
    auto fail = [&](const char* what) {
        cleanup();
        set_error("cell structures: %s", what);
        return RTT_ECUDA;
    };
    if (cudaMalloc(&keys_out, E * 4) != cudaSuccess || cudaMalloc(&vals_in, E * 4) != cudaSuccess ||
        cudaMalloc(&cray, E * 4) != cudaSuccess)
        return fail("allocation");
    std::vector<int32_t> seq(E);
    for (int64_t e = 0; e < E; ++e) seq[e] = (int32_t)e;
    if (cudaMemcpyAsync(vals_in, seq.data(), E * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail("copy");
    if (cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, op->node00, keys_out, vals_in, cray, E, 0,
                                        end_bit, st) != cudaSuccess ||
        cudaMalloc(&tmp, tmp_bytes) != cudaSuccess ||
        cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, op->node00, keys_out, vals_in, cray, E, 0,
                                        end_bit, st) != cudaSuccess)
        return fail("sort");
    // ray tables in cell order
    cudaError_t e2 = cudaSuccess;
    auto dev = [&](auto** d, size_t n) {
        if (e2 == cudaSuccess) e2 = cudaMalloc((void**)d, n * sizeof(**d) + 16);
    };
    dev(&op->c_row, E);
    dev(&op->c_col, E);
    dev(&op->c_K0, E);
    dev(&op->c_F0, E);
    dev(&op->c_fb, E);
    dev(&op->c_r0, E);
    dev(&op->c_W, E);
    dev(&op->c_W64, 4 * E);
    dev(&op->c_F64, E);
    if (e2 != cudaSuccess) return fail("allocation of the cell-ordered tables");
    cell_tables<<<(unsigned)((E + 255) / 256), 256, 0, st>>>(
        E, n_phi, frames_per_hat(op->frame_D), op->frame_D, cray, op->ray_row, op->node00, op->K0,
        op->F0, op->W, op->W64, op->F64, op->c_row, op->c_col, op->c_K0, op->c_F0, op->c_fb,
        op->c_r0, op->c_W, op->c_W64, op->c_F64);
    if (cudaGetLastError() != cudaSuccess) return fail("table kernel");
    std::vector<int32_t> cell(E);
    if (cudaMemcpyAsync(cell.data(), keys_out, E * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail("copy back");
    cleanup();
    // rays per cell and the first sorted position of each cell
    std::vector<int64_t> cstart(n_cells + 1, 0);
    for (int64_t e = 0; e < E; ++e) {
        const int c = cell[e];
        if (c < 0 || c >= n_cells) return fail("ray outside the cell range");
        ++cstart[c + 1];
    }
    for (int64_t c = 0; c < n_cells; ++c) cstart[c + 1] += cstart[c];
    // strip segments: consecutive columns, at most kSegMaxCols of them and at
    // most kSegMaxRays rays unless one column alone has more
    std::vector<int32_t> s_ray, s_col, s_ncol, s_rec;
    std::vector<int32_t> seg_of((size_t)n_cells);  // cell -> segment
    int64_t rec = 0;
    for (int i = 0; i < n_strips; ++i) {
        int j = 0;
        while (j < n_phi) {
            const int64_t c0 = (int64_t)i * n_phi + j;
            int64_t rays = cstart[c0 + 1] - cstart[c0];
            int nc = 1;
            while (j + nc < n_phi && nc < kSegMaxCols) {
                const int64_t cn = c0 + nc;
                const int64_t add = cstart[cn + 1] - cstart[cn];
                if (rays + add > kSegMaxRays) break;
                rays += add;
                ++nc;
            }
            const int sg = (int)s_col.size();
            for (int q = 0; q < nc; ++q) seg_of[c0 + q] = sg;
            s_ray.push_back((int32_t)cstart[c0]);
            s_col.push_back(j);
            s_ncol.push_back(nc);
            s_rec.push_back((int32_t)rec);
            rec += 2 * (nc + 1);
            j += nc;
        }
    }
    const int n_seg = (int)s_col.size();
    s_ray.push_back((int32_t)E);
    if (rec >= (int64_t)1 << 31) return fail("too many partial records");
    // gather table: per node (i, j) the records of strip i - 1 (upper row) and
    // strip i (lower row), each from the segment before (if column j starts
    // its segment) and from the own segment; -1 where none
    std::vector<int32_t> gs((size_t)S * 4, -1);
    for (int i = 0; i < n_r; ++i)
        for (int j = 0; j < n_phi; ++j) {
            int32_t* o = &gs[((size_t)i * n_phi + j) * 4];
            for (int half = 1; half >= 0; --half) {
                const int strip = half ? i - 1 : i;
                if (strip < 0 || strip >= n_strips) continue;
                const int own = seg_of[(size_t)strip * n_phi + j];
                const int prev = seg_of[(size_t)strip * n_phi + (j + n_phi - 1) % n_phi];
                int32_t* q = o + (half ? 0 : 2);
                // column j is the successor column of the segment before it
                if (j == s_col[own]) q[0] = s_rec[prev] + 2 * s_ncol[prev] + half;
                q[1] = s_rec[own] + 2 * (j - s_col[own]) + half;
            }
        }
    auto up = [&](int32_t** d, const std::vector<int32_t>& h) {
        if (e2 != cudaSuccess) return;
        e2 = cudaMalloc(d, h.size() * 4 + 16);
        if (e2 == cudaSuccess) e2 = cudaMemcpy(*d, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
    };
    up(&op->seg_ray, s_ray);
    up(&op->seg_col, s_col);
    up(&op->seg_ncol, s_ncol);
    up(&op->seg_rec, s_rec);
    up(&op->gslot, gs);
    {
        std::vector<int32_t> cp(cstart.size());
        for (size_t c = 0; c < cstart.size(); ++c) cp[c] = (int32_t)cstart[c];
        up(&op->cell_ptr, cp);
    }
    if (e2 == cudaSuccess) e2 = cudaMalloc(&op->adj_ctr, 16);
    if (e2 == cudaSuccess) e2 = cudaMemset(op->adj_ctr, 0, 16);
    if (e2 != cudaSuccess) return fail("upload");
    op->n_seg = n_seg;
    op->n_rec = rec;
    return RTT_OK;
}

static CellArgs cell_args(const rtt_op_s* op, const void* y, int B, const ArmSeg& seg) {
    CellArgs a{};
    a.c_row = op->c_row;
    a.c_col = op->c_col;
    a.c_h0 = op->c_K0;
    a.c_h1 = op->c_F0;
    a.c_W = op->c_W;
    a.c_W16 = op->c_W16;
    a.c_W64 = op->c_W64;
    a.c_F64 = op->c_F64;
    a.seg_ray = op->seg_ray;
    a.seg_col = op->seg_col;
    a.seg_ncol = op->seg_ncol;
    a.seg_rec = op->seg_rec;
    a.seg = seg;
    a.seg_rows_all = (int)op->n_rows;
    a.K = op->time.n_hats;
    a.Tn = op->time.n_frames;
    a.B = B;
    a.D = (int32_t)op->frame_D;
    a.ctr = op->adj_ctr;
    a.status = op->dev_status;
    a.y = y;
    a.part = op->cpart;
    return a;
}

// whether the TMA kernel serves this call (FP32, whole batch one chunk)
static bool tma_shape(const rtt_op_s* op, int B, int P, int* hg) {
    if (P == 0 || !(B == 4 || B == 8 || B == 16)) return false;
    const int F = 32 / B;
    if (P % F != 0 || op->time.n_frames % F != 0) return false;
    *hg = B <= 8 ? 2 : 1;
    const int rows = ((32 * *hg + 1) * P + 2 * (F - 1)) / F;
    return rows <= 256;
}

template <int BC, int P, int HG>
static cudaError_t launch_cell_tma(CellArgs a, const float* y, const int32_t* op_fb,
                                   const int32_t* op_r0, cudaStream_t st) {
    constexpr int F = CellBox<BC, P, HG>::kF;
    constexpr int ROWS = CellBox<BC, P, HG>::kRows;
    static_assert(ROWS <= 256, "TMA box rows");
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || a.seg.total <= 0 || ((uintptr_t)y % 16) != 0 || a.B != BC || a.Tn % F != 0)
        return cudaErrorNotSupported;
    CUtensorMap m;
    // (32 floats = one 128-byte line, lines of a data row's frames, data rows)
    cuuint64_t dims[3] = {32, (cuuint64_t)(a.Tn / F), (cuuint64_t)a.seg.total};
    cuuint64_t strides[2] = {128, (cuuint64_t)(a.Tn / F) * 128};
    cuuint32_t box[3] = {32, (cuuint32_t)ROWS, 1};
    cuuint32_t es[3] = {1, 1, 1};
    if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(y), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    a.n_hg = (a.K + 32 * HG - 1) / (32 * HG);
    a.n_bc = 1;
    a.hw = 32 * HG;
    a.c_h0 = op_fb;  // the periodic tap tables (cell_tables)
    a.c_h1 = op_r0;
    a.n_items = (int64_t)a.n_hg * a.n_items;  // n_items holds the segment count on entry
    const size_t smem = 1024 + (size_t)kCellWarps * 2 * CellBox<BC, P, HG>::kStride + kCellWarps * 16;
    cudaError_t e = cudaFuncSetAttribute(adj_cell_tma_kernel<BC, P, HG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid =
        resident_grid(adj_cell_tma_kernel<BC, P, HG>, kCellWarps * 32, smem, a.n_items, kCellWarps);
    return launch_dependent(adj_cell_tma_kernel<BC, P, HG>, dim3(grid), dim3(kCellWarps * 32), smem, st,
                            m, a);
}

static cudaError_t dispatch_tma(const rtt_op_s* op, const CellArgs& a, const float* y, int B, int P,
                                int hg, cudaStream_t st) {
    const int32_t *fb = op->c_fb, *r0 = op->c_r0;
    if (B == 4 && P == 8)
        return hg == 2 ? launch_cell_tma<4, 8, 2>(a, y, fb, r0, st) : launch_cell_tma<4, 8, 1>(a, y, fb, r0, st);
    if (B == 8 && P == 4)
        return hg == 2 ? launch_cell_tma<8, 4, 2>(a, y, fb, r0, st) : launch_cell_tma<8, 4, 1>(a, y, fb, r0, st);
    if (B == 8 && P == 8)
        return hg == 2 ? launch_cell_tma<8, 8, 2>(a, y, fb, r0, st) : launch_cell_tma<8, 8, 1>(a, y, fb, r0, st);
    if (B == 16 && P == 2) return launch_cell_tma<16, 2, 1>(a, y, fb, r0, st);
    if (B == 16 && P == 4) return launch_cell_tma<16, 4, 1>(a, y, fb, r0, st);
    if (B == 16 && P == 8) return launch_cell_tma<16, 8, 1>(a, y, fb, r0, st);
    return cudaErrorNotSupported;
}

// one 32- or 64-column pass through adj_cell_tma_pass_kernel;
// cudaErrorNotSupported unless the pass has PW columns of a batch of whole
// passes and the periodic cadence P in {2, 4, 8}
template <int PW, int P>
static cudaError_t launch_cell_tma_pass(CellArgs a, const float* y, const int32_t* op_fb,
                                        const int32_t* op_r0, cudaStream_t st) {
    using Box = CellBoxPass<PW, P>;
    static_assert(Box::kFrames <= 256, "TMA box rows");
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    const float* yp = y + a.b0;
    if (!enc || a.seg.total <= 0 || a.Bp != PW || a.B % PW != 0 || ((uintptr_t)yp % 16) != 0)
        return cudaErrorNotSupported;
    CUtensorMap m;
    CUresult r;
    cuuint32_t es[4] = {1, 1, 1, 1};
    if constexpr (Box::kG == 1) {
        // (the pass's 32 floats = one 128-byte line, frames of a data row, data rows)
        cuuint64_t dims[3] = {32, (cuuint64_t)a.Tn, (cuuint64_t)a.seg.total};
        cuuint64_t strides[2] = {(cuuint64_t)a.B * 4, (cuuint64_t)a.Tn * a.B * 4};
        cuuint32_t box[3] = {32, (cuuint32_t)Box::kFrames, 1};
        r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(yp), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        // (32 floats = one 128-byte line, the pass's two lines of a frame, frames, data rows)
        cuuint64_t dims[4] = {32, 2, (cuuint64_t)a.Tn, (cuuint64_t)a.seg.total};
        cuuint64_t strides[3] = {128, (cuuint64_t)a.B * 4, (cuuint64_t)a.Tn * a.B * 4};
        cuuint32_t box[4] = {32, 2, (cuuint32_t)Box::kFrames, 1};
        r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(yp), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return cudaErrorNotSupported;
    a.n_hg = (a.K + Box::kW - 1) / Box::kW;
    a.n_bc = 1;
    a.hw = Box::kW;
    a.c_h0 = op_fb;  // the periodic tap tables (cell_tables)
    a.c_h1 = op_r0;
    a.n_items = (int64_t)a.n_hg * a.n_items;  // n_items holds the segment count on entry
    const size_t smem = 1024 + (size_t)kCellWarps * 2 * Box::kStride + kCellWarps * 16;
    auto kern = adj_cell_tma_pass_kernel<PW, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = resident_grid(kern, kCellWarps * 32, smem, a.n_items, kCellWarps);
    return launch_dependent(kern, dim3(grid), dim3(kCellWarps * 32), smem, st, m, a);
}

static cudaError_t dispatch_tma_pass(const rtt_op_s* op, const CellArgs& a, const float* y, int P,
                                     cudaStream_t st) {
    const int32_t *fb = op->c_fb, *r0 = op->c_r0;
    if (a.Bp == 64) {
        switch (P) {
            case 2: return launch_cell_tma_pass<64, 2>(a, y, fb, r0, st);
            case 4: return launch_cell_tma_pass<64, 4>(a, y, fb, r0, st);
            case 8: return launch_cell_tma_pass<64, 8>(a, y, fb, r0, st);
            default: return cudaErrorNotSupported;
        }
    }
    switch (P) {
        case 2: return launch_cell_tma_pass<32, 2>(a, y, fb, r0, st);
        case 4: return launch_cell_tma_pass<32, 4>(a, y, fb, r0, st);
        case 8: return launch_cell_tma_pass<32, 8>(a, y, fb, r0, st);
        default: return cudaErrorNotSupported;
    }
}

// a 1- or 2-column batch through adj_cell_direct_kernel; cudaErrorNotSupported
// unless the cadence is periodic (P in {2, 4, 8})
template <int BC, int P, int HG>
static cudaError_t launch_cell_direct(CellArgs a, const int32_t* op_fb, const int32_t* op_r0,
                                      cudaStream_t st) {
    if (a.seg.total <= 0 || a.B != BC || a.Bp != BC) return cudaErrorNotSupported;
    a.n_hg = (a.K + 32 * HG - 1) / (32 * HG);
    a.n_bc = 1;
    a.hw = 32 * HG;
    a.c_h0 = op_fb;  // the periodic tap tables (cell_tables)
    a.c_h1 = op_r0;
    a.n_items = (int64_t)a.n_hg * a.n_items;  // n_items holds the segment count on entry
    const int grid =
        resident_grid(adj_cell_direct_kernel<BC, P, HG>, kCellWarps * 32, 0, a.n_items, kCellWarps);
    return launch_dependent(adj_cell_direct_kernel<BC, P, HG>, dim3(grid), dim3(kCellWarps * 32), 0, st,
                            a);
}

static cudaError_t dispatch_direct(const rtt_op_s* op, const CellArgs& a, int B, int P, int hg,
                                   cudaStream_t st) {
    const int32_t *fb = op->c_fb, *r0 = op->c_r0;
    auto go = [&](auto b_tag, auto p_tag) -> cudaError_t {
        constexpr int BC = decltype(b_tag)::value, PP = decltype(p_tag)::value;
        return hg == 2 ? launch_cell_direct<BC, PP, 2>(a, fb, r0, st)
                       : launch_cell_direct<BC, PP, 1>(a, fb, r0, st);
    };
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I4 = std::integral_constant<int, 4>;
    using I8 = std::integral_constant<int, 8>;
    if (B == 1) {
        if (P == 2) return go(I1{}, I2{});
        if (P == 4) return go(I1{}, I4{});
        if (P == 8) return go(I1{}, I8{});
    } else if (B == 2) {
        if (P == 2) return go(I2{}, I2{});
        if (P == 4) return go(I2{}, I4{});
        if (P == 8) return go(I2{}, I8{});
    }
    return cudaErrorNotSupported;
}

// staged-frame capacity of the general kernel's buffers
constexpr int kGenFrameCap = 192;

template <typename T, int BC>
static cudaError_t launch_cell_gen_bc(CellArgs a, cudaStream_t st) {
    constexpr int E = BC * (int)sizeof(T);
    const int64_t D = a.D;
    // hats per item: the frames of (hw + 1) hat steps must fit the buffer
    int64_t hw = ((int64_t)(kGenFrameCap - 2) * D) / kFracOne - 1;
    if (hw > 32) hw = 32;
    if (hw < 1) hw = 1;
    a.hw = (int)hw;
    a.fwin = (int)((((int64_t)(hw + 1) * kFracOne) + D - 1) / D) + 1;
    const uint32_t buf = (uint32_t)(((size_t)stage_off(a.fwin, E) + 16 + 15) & ~(size_t)15);
    const size_t smem = (size_t)kGenWarps * 2 * buf;
    if (smem > 200 * 1024) return cudaErrorNotSupported;  // cadence far finer than any hat step in use
    a.n_hg = (int)((a.K + hw - 1) / hw);
    a.n_bc = (a.Bp + BC - 1) / BC;
    a.n_items = a.n_items * a.n_hg * a.n_bc;  // n_items holds the segment count on entry
    const int vec = (E % 16 == 0) && ((a.B * (int)sizeof(T)) % 16 == 0) &&
                    ((a.b0 * (int)sizeof(T)) % 16 == 0) && (a.Bp % BC == 0) &&
                    ((uintptr_t)a.y % 16 == 0);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(adj_cell_gen_kernel<T, BC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid =
        resident_grid(adj_cell_gen_kernel<T, BC>, kGenWarps * 32, smem, a.n_items, kGenWarps);
    return launch_dependent(adj_cell_gen_kernel<T, BC>, dim3(grid), dim3(kGenWarps * 32), smem, st, a,
                            buf, vec);
}

template <typename T, int BC, int P, int NH>
static cudaError_t launch_cell_per(CellArgs a, const int32_t* fb, const int32_t* r0, cudaStream_t st) {
    constexpr int E = BC * (int)sizeof(T);
    a.hw = 32 * NH;
    a.fwin = (32 * NH + 1) * P;
    const uint32_t buf = (uint32_t)(((size_t)stage_off(a.fwin, E) + 16 + 15) & ~(size_t)15);
    const size_t smem = (size_t)kGenWarps * 2 * buf;
    if (smem > 200 * 1024) return cudaErrorNotSupported;
    a.n_hg = (a.K + 32 * NH - 1) / (32 * NH);
    a.n_bc = (a.Bp + BC - 1) / BC;
    a.n_items = a.n_items * a.n_hg * a.n_bc;  // n_items holds the segment count on entry
    a.c_h0 = fb;
    a.c_h1 = r0;
    const int vec = (E % 16 == 0) && ((a.B * (int)sizeof(T)) % 16 == 0) &&
                    ((a.b0 * (int)sizeof(T)) % 16 == 0) && (a.Bp % BC == 0) &&
                    ((uintptr_t)a.y % 16 == 0);
    auto kern = adj_cell_per_kernel<T, BC, P, NH>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = resident_grid(kern, kGenWarps * 32, smem, a.n_items, kGenWarps);
    return launch_dependent(kern, dim3(grid), dim3(kGenWarps * 32), smem, st, a, buf, vec);
}

// the periodic staged kernel: 8-column chunks (FP32) or 4-column chunks (FP64),
// two hats per lane; cudaErrorNotSupported for other cadences
template <typename T>
static cudaError_t launch_cell_per_any(const rtt_op_s* op, const CellArgs& a, cudaStream_t st) {
    const int P = frames_per_hat(op->frame_D);
    const int32_t *fb = op->c_fb, *r0 = op->c_r0;
    if constexpr (sizeof(T) == 4) {
        if (a.Bp % 16 == 0) {  // 64-byte pieces of each frame record
            if (P == 2) return launch_cell_per<T, 16, 2, 1>(a, fb, r0, st);
            if (P == 4) return launch_cell_per<T, 16, 4, 1>(a, fb, r0, st);
            if (P == 8) return launch_cell_per<T, 16, 8, 1>(a, fb, r0, st);
        } else if (a.Bp % 8 == 0) {
            if (P == 2) return launch_cell_per<T, 8, 2, 2>(a, fb, r0, st);
            if (P == 4) return launch_cell_per<T, 8, 4, 2>(a, fb, r0, st);
            if (P == 8) return launch_cell_per<T, 8, 8, 2>(a, fb, r0, st);
        } else {
            if (P == 2) return launch_cell_per<T, 4, 2, 2>(a, fb, r0, st);
            if (P == 4) return launch_cell_per<T, 4, 4, 2>(a, fb, r0, st);
            if (P == 8) return launch_cell_per<T, 4, 8, 2>(a, fb, r0, st);
        }
    } else {
        if (P == 2) return launch_cell_per<T, 4, 2, 1>(a, fb, r0, st);
        if (P == 4) return launch_cell_per<T, 4, 4, 1>(a, fb, r0, st);
        if (P == 8) return launch_cell_per<T, 4, 8, 1>(a, fb, r0, st);
    }
    return cudaErrorNotSupported;
}

template <typename T>
static cudaError_t launch_cell_gen(const CellArgs& a, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (a.Bp >= 8) return launch_cell_gen_bc<T, 8>(a, st);
        if (a.Bp >= 4) return launch_cell_gen_bc<T, 4>(a, st);
        if (a.Bp >= 2) return launch_cell_gen_bc<T, 2>(a, st);
        return launch_cell_gen_bc<T, 1>(a, st);
    } else {
        if (a.Bp >= 4) return launch_cell_gen_bc<T, 4>(a, st);
        if (a.Bp >= 2) return launch_cell_gen_bc<T, 2>(a, st);
        return launch_cell_gen_bc<T, 1>(a, st);
    }
}

template <typename T>
static cudaError_t launch_gather(const rtt_op_s* op, T* x, int B, int b0, int Bp, cudaStream_t st) {
    const int64_t S = op->n_nodes;
    const int K = op->time.n_hats;
    const int sms = sm_count();
    if constexpr (sizeof(T) == 4) {
        if (Bp % 4 == 0 && B % 4 == 0 && b0 % 4 == 0 && ((uintptr_t)x % 16) == 0) {
            const int64_t n = S * K * Bp / 4;
            const int64_t want = (n + 255) / 256;
            const int grid = (int)(want < (int64_t)sms * 8 ? (want > 0 ? want : 1) : (int64_t)sms * 8);
            return launch_dependent(adj_gather4_kernel, dim3(grid), dim3(256), 0, st,
                                    (const int32_t*)op->gslot, (const float*)op->cpart, (float*)x, S, K,
                                    B, b0, Bp, op->adj_ctr);
        }
    }
    const int64_t n = S * K * Bp;
    const int64_t want = (n + 255) / 256;
    const int grid = (int)(want < (int64_t)sms * 8 ? (want > 0 ? want : 1) : (int64_t)sms * 8);
    return launch_dependent(adj_gather_kernel<T>, dim3(grid), dim3(256), 0, st,
                            (const int32_t*)op->gslot, (const T*)op->cpart, x, S, K, B, b0, Bp,
                            op->adj_ctr);
}

// the adjoint kernel an FP32 call of `batch` columns can use at most:
// 4 (TMA, 64-hat items), 3 (TMA, 32-hat items), 2 (periodic, staged by
// per-lane copies) or 1 (general)
int adjoint_best_kind(const rtt_op_s* op, int batch) {
    const int P = frames_per_hat(op->frame_D);
    int hg = 0;
    if (tma_shape(op, batch, P, &hg)) return hg == 2 ? 4 : 3;
    if (P > 0 && batch % 32 == 0) return 4;  // 32- or 64-column passes by the TMA kernel
    if (P > 0 && batch <= 2) return 4;       // the direct-load kernel (kinds 3 and 4: 32- or 64-hat items)
    return P > 0 ? 2 : 1;
}

template <typename T>
cudaError_t launch_adjoint(const rtt_op_s* op, const T* y, T* x, int B, const ArmSeg& seg,
                           cudaStream_t st) {
    const int K = op->time.n_hats;
    if (seg.total == 0)  // no data rows in the arm: A^T y = 0
        return cudaMemsetAsync(x, 0, (size_t)op->n_nodes * K * B * sizeof(T), st);
    if (!op->cpart || op->cpart_bytes < adjoint_scratch_bytes(op, B, (int)sizeof(T))) {
        set_error("adjoint scratch not prepared for batch %d", B);
        return cudaErrorInvalidValue;
    }
    int PC = pass_cols((int)sizeof(T), B);
    int kind = frames_per_hat(op->frame_D) > 0 ? 2 : 1;  // FP64: periodic when the cadence allows
    if constexpr (sizeof(T) == 4) {
        const ApplyVariant v = variant_for(op, B);
        kind = v.adj;
        const int best = adjoint_best_kind(op, B);
        if (kind > best) kind = best;
        if (v.adj_cols > 0 && v.adj_cols < PC) PC = v.adj_cols;
    }
    for (int b0 = 0; b0 < B; b0 += PC) {
        const int Bp = B - b0 < PC ? B - b0 : PC;
        CellArgs a = cell_args(op, y, B, seg);
        a.b0 = b0;
        a.Bp = Bp;
        a.n_items = op->n_seg;
        cudaError_t e = cudaErrorNotSupported;
        if constexpr (sizeof(T) == 4) {
            if (kind >= 3 && B <= 2)
                e = dispatch_direct(op, a, B, frames_per_hat(op->frame_D), kind == 4 ? 2 : 1, st);
            else if (kind >= 3 && Bp == B && B <= 16)
                e = dispatch_tma(op, a, (const float*)y, B, frames_per_hat(op->frame_D), kind == 4 ? 2 : 1,
                                 st);
            else if (kind >= 3 && (Bp == 32 || Bp == 64) && B % Bp == 0)
                e = dispatch_tma_pass(op, a, (const float*)y, frames_per_hat(op->frame_D), st);
        }
        if (e == cudaErrorNotSupported && kind >= 2) {
            cudaGetLastError();  // clear the "not supported" marker, if any
            e = launch_cell_per_any<T>(op, a, st);
        }
        if (e == cudaErrorNotSupported) {
            cudaGetLastError();
            e = launch_cell_gen<T>(a, st);
        }
        if (e != cudaSuccess) return e;
        e = launch_gather<T>(op, x, B, b0, Bp, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t launch_adjoint<float>(const rtt_op_s*, const float*, float*, int, const ArmSeg&,
                                          cudaStream_t);
template cudaError_t launch_adjoint<double>(const rtt_op_s*, const double*, double*, int,
                                           const ArmSeg&, cudaStream_t);

}  // namespace rtt
