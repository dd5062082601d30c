// Internal definitions shared by the librtt translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "rtt.h"

// return the status of x from the calling function unless it is RTT_OK
#define RTT_TRY(x)                   \
    do {                             \
        rtt_status _s = (x);         \
        if (_s != RTT_OK) return _s; \
    } while (0)

namespace rtt {

// 24 fractional bits for the per-ray hat offset: the fraction of every
// (ray, frame) sample is then an exact FP32 value and the hat index is an
// exact integer computation.
constexpr int kFracBits = 24;
constexpr int32_t kFracOne = 1 << kFracBits;
constexpr int32_t kFracMask = kFracOne - 1;

void set_error(const char* fmt, ...);

struct ArmSeg;

// Rows selected by an arm mask: up to three contiguous segments of the
// (order, pixel)-sorted row list, concatenated in order.
struct ArmSeg {
    int32_t begin[3];   // first input row of segment
    int32_t len[3];     // number of rows
    int32_t out_off[3]; // first output row of segment
    int32_t n;          // number of segments
    int32_t total;      // total selected rows
    int32_t mask;
};

rtt_status make_seg(const struct ::rtt_op_s* op, int mask, ArmSeg* s);

// Kernel variants of one FP32 apply.  Every variant sums each output in the
// same order with the same fused multiply-adds, so the choice changes speed
// only, never a bit of the result.
struct ApplyVariant {
    int8_t fwd = 0;     // forward: 1 staged z (fwd3), 2 lane-per-hat shuffles (fwd4),
                        // 3 TMA corner slabs (fwd5), 4 pipelined bulk corner copies
                        // (fwd6), 5 periodic one-chunk staged (fwd7), 6 the same with its
                        // table loads one task ahead (fwd8), 7 periodic quad-lane (fwd9),
                        // 8 the same with its table loads one task ahead, 9 quad-lane with
                        // the corner slabs staged one ray ahead (fwd10)
    int8_t fwd_bc = 0;  // batch entries per forward task (power of two)
    int8_t fwd_half = 0; // staged forward: half the frames per lane (fewer registers)
    int8_t fwd_su = 2;   // staged forward: staging items in flight per lane (1, 2 or 3)
    int8_t fwd_order = 0; // forward task rows: 0 (order, pixel), 1 source-cell order
    int8_t fwd_cols = 0;  // periodic forward: 0 all columns at once, else passes of this many
    int8_t adj_cols = 0;  // adjoint: columns per pass (0: 32 in FP32, 16 in FP64)
    int8_t adj = 0;     // adjoint: 1 general, 2 periodic staged by per-lane copies, 3 TMA
                        // with 32-hat items, 4 TMA with 64-hat items (the most the call allows)
};
constexpr int kMaxTuned = 8;  // batch sizes with an autotuned variant per operator

// the variant an FP32 apply of `batch` columns uses: the tuned one if
// rtt_autotune ran for that batch size, else the default rule
ApplyVariant variant_for(const struct ::rtt_op_s* op, int batch);

}  // namespace rtt

struct rtt_op_s {
    rtt_geometry geom;
    rtt_source_grid grid;
    rtt_time_grid time;
    rtt_options opt;
    int64_t n_rays = 0;
    int64_t n_rows = 0;
    // row shard (rtt_build_operator_shard): this operator holds rows
    // [shard_row_begin, shard_row_begin + n_rows) of the whole table's total_rows
    int64_t total_rows = 0;
    int64_t total_row_begin[4] = {0, 0, 0, 0};  // row_begin of the whole table
    int64_t shard_row_begin = 0;
    int32_t shard_index = 0;
    int32_t shard_count = 1;
    int64_t row_begin[4] = {0, 0, 0, 0};  // rows of order n: [row_begin[n], row_begin[n+1])
    int32_t n_nodes = 0;
    int64_t frame_D = 0;  // (cadence / hat_step) * 2^24, exact integer
    double delta = 0.0;   // cadence / hat_step
    double s_ref = 0.0, scale = 0.0;
    double dmin[3], dmax[3];

    // rays sorted by row (device)
    int32_t* row_ptr = nullptr;   // [R+1]
    int32_t* ray_row = nullptr;   // [E]
    int32_t* node00 = nullptr;    // [E] node (i0, j0)
    int32_t* node01 = nullptr;    // [E] node (i0, j1), j1 = (j0 + 1) mod n_phi
    float4* W = nullptr;          // [E] scale * w * bilinear, corners (i0j0, i1j0, i0j1, i1j1)
    double* W64 = nullptr;        // [4E] same in FP64
    uint2* W16 = nullptr;         // [E] BF16 copy of W when the weights are BF16 (else null)
    int weight_precision = 0;     // RTT_WEIGHTS_FP32 or RTT_WEIGHTS_BF16
    int32_t* K0 = nullptr;        // [E] floor(u0)
    int32_t* F0 = nullptr;        // [E] floor(frac(u0) * 2^24)
    float4* ray_rec = nullptr;    // [2E] a ray's forward fields in one 32-byte record:
                                  // (K0, F0, node00, node01) as int bits, then W
    double* F64 = nullptr;        // [E] frac(u0) exactly
    double* r = nullptr;          // [E] FP64 copies for probes and quantiles
    double* phi = nullptr;        // [E] source azimuth (localized probes)
    double* delay = nullptr;
    double* weight = nullptr;
    double* thr = nullptr;
    int32_t* row_order = nullptr; // [R] order of each row
    int32_t* row_pixel = nullptr; // [R] pixel of each row
    int32_t* row_sched = nullptr; // [R] rows by source cell (Morton order of the first ray's
                                  // cell) within each order: the forward's alternative task order
    // adjoint by source cells (adjoint.cu): ray tables in cell order, strip
    // segments of cells, their partial records and the gather table
    int32_t* c_row = nullptr;    // [E] input data row
    int32_t* c_col = nullptr;    // [E] cell column
    int32_t* c_K0 = nullptr;     // [E]
    int32_t* c_F0 = nullptr;     // [E]
    int32_t* c_fb = nullptr;     // [E] periodic cadences: first tap frame of hat 0
    int32_t* c_r0 = nullptr;     // [E] periodic cadences: tap weight phase
    float4* c_W = nullptr;       // [E]
    uint2* c_W16 = nullptr;      // [E] BF16 copy of c_W, or null
    double* c_W64 = nullptr;     // [4E]
    double* c_F64 = nullptr;     // [E]
    int32_t* seg_ray = nullptr;  // [n_seg + 1]
    int32_t* seg_col = nullptr;  // [n_seg]
    int32_t* seg_ncol = nullptr; // [n_seg]
    int32_t* seg_rec = nullptr;  // [n_seg]
    int32_t* gslot = nullptr;    // [S][4] records of each node, -1 for none
    int32_t* cell_ptr = nullptr; // [cells + 1] first cell-ordered ray of each cell (i0 n_phi + j0)
    int32_t n_seg = 0;
    int64_t n_rec = 0;
    int* adj_ctr = nullptr;      // work ticket counter of the adjoint (reset by its gather)
    void* cpart = nullptr;       // partial records [n_rec][K][<= 32 columns], grown on demand
    size_t cpart_bytes = 0;
    void* rscratch = nullptr;  // residual y - d of the separate-path rtt_apply_A_AT, grown on demand
    size_t rscratch_bytes = 0;
    int* dev_status = nullptr;  // device status word: bit 0 = a kernel's bounded wait timed out
    // order mixing (Eq. 4), built on first use for one arm mask: the arm's
    // output rows grouped by pixel (unresolved image), and the scratch of the
    // total-flux row reduction
    struct MixGroups {
        int arm_mask = -1;
        int32_t n_groups = 0;
        int32_t* grp_ptr = nullptr;   // [G+1] into grp_rows
        int32_t* grp_rows = nullptr;  // arm output rows, pixel-major, orders ascending
        int32_t* row_grp = nullptr;   // [arm rows] group of each row
        float* inv32 = nullptr;       // [G] 1 / sqrt(rows in group), FP32
        double* inv64 = nullptr;      // [G] the same in FP64
        void* part = nullptr;         // total-flux partial sums, grown on demand
        size_t part_bytes = 0;
    } mix;
    // autotuned kernel variants (rtt_autotune), per batch size
    int n_tuned = 0;
    int tuned_batch[rtt::kMaxTuned] = {};
    rtt::ApplyVariant tuned[rtt::kMaxTuned];
};

namespace rtt {
// RTT_ESTATE for a row shard at entry points that need every row of the
// operator (order mixing, quantiles, reach, audit, solvers)
inline rtt_status whole_only(const rtt_op_s* op, const char* what) {
    if (op && op->shard_count > 1) {
        set_error("%s needs the whole operator (this is row shard %d of %d)", what,
                  op->shard_index, op->shard_count);
        return RTT_ESTATE;
    }
    return RTT_OK;
}

// order mixing (mix.cu): pixel groups of an arm, mixed row count, and the
// collapse (adjoint = false: arm rows -> mixed rows) or its adjoint over
// `cols` = n_frames * batch values per row
rtt_status mix_prepare(rtt_op_s* op, const ArmSeg& seg);
int64_t mix_out_rows(const rtt_op_s* op, const ArmSeg& seg, int mode);
template <typename T>
rtt_status launch_mix(rtt_op_s* op, const ArmSeg& seg, int mode, const T* in, T* out, int64_t cols,
                      bool adjoint, cudaStream_t st);
// the adjoint's partial-record scratch for `batch` columns of `elem`-byte
// values (grown on demand; synchronises the device when it grows)
rtt_status ensure_adjoint_scratch(rtt_op_s* op, int batch, int elem);
size_t adjoint_scratch_bytes(const rtt_op_s* op, int batch, int elem);
rtt_status build_cells(rtt_op_s* op, cudaStream_t st);
template <typename T>
cudaError_t launch_adjoint(const rtt_op_s* op, const T* y, T* x, int B, const ArmSeg& seg,
                           cudaStream_t st);
template <typename T>
cudaError_t launch_forward(const rtt_op_s* op, const T* x, T* y, int B, const ArmSeg& seg,
                           cudaStream_t st);

// batched audit stages (one launch per stage over all (operator, arm) jobs;
// buffers allocated at create, no host synchronisation in a run)
struct ProbePlan;
rtt_status probe_plan_create(const rtt_op_s* const* job_ops, const ArmSeg* segs, int n_jobs, int n_ages,
                             const double* ages_host, double h, ProbePlan** out);
cudaError_t probe_plan_run(ProbePlan* pp, cudaStream_t st);
const double* probe_plan_info(const ProbePlan* pp);  // device [jobs][ages]
void probe_plan_destroy(ProbePlan* pp);
struct ClassPlan;
rtt_status class_plan_create(const rtt_op_s* const* ops, int n_ops, const int* job_op, const ArmSeg* segs,
                             int n_jobs, int kind, double* G, cudaStream_t st, ClassPlan** out);
cudaError_t class_plan_run(ClassPlan* cp, cudaStream_t st);
void class_plan_destroy(ClassPlan* cp);
cudaError_t launch_eigvals_batched(int n, int batch, double* A, double* d, double* e, double* work,
                                   double* ev, cudaStream_t st);
}  // namespace rtt
