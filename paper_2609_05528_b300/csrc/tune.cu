// Autotuner for the FP32 applies: for one operator and batch size, times
// every kernel variant of the forward (staged, lane-per-hat or quad-lane,
// batch entries and frames per task) and of the adjoint (frames staged by per-lane copies
// or by TMA tensor copies, 32- or 64-hat items) with CUDA events on the
// caller's stream, and records the fastest in the operator.  All variants
// produce the same bits (same per-output summation order and fused
// multiply-adds), so tuning changes speed only.
#include <cuda_runtime.h>

#include <vector>

#include "rtt_internal.cuh"

using namespace rtt;

namespace rtt {
int adjoint_best_kind(const rtt_op_s* op, int batch);
}  // namespace rtt

namespace {

constexpr int kTuneReps = 3;

// a candidate replaces the best so far only when it is at least 1% faster:
// near-ties (run-to-run noise) keep the earlier, simpler choice, so the
// tuner picks the same variant from run to run
inline bool better(float ms, float best) { return ms < 0.99f * best; }

// installs v as the operator's variant for batch B (replacing an entry)
void set_variant(rtt_op_s* op, int B, const ApplyVariant& v) {
    for (int i = 0; i < op->n_tuned; ++i)
        if (op->tuned_batch[i] == B) {
            op->tuned[i] = v;
            return;
        }
    int slot = op->n_tuned < kMaxTuned ? op->n_tuned++ : kMaxTuned - 1;
    op->tuned_batch[slot] = B;
    op->tuned[slot] = v;
}

void clear_variant(rtt_op_s* op, int B) {
    for (int i = 0; i < op->n_tuned; ++i)
        if (op->tuned_batch[i] == B) {
            for (int j = i + 1; j < op->n_tuned; ++j) {
                op->tuned_batch[j - 1] = op->tuned_batch[j];
                op->tuned[j - 1] = op->tuned[j];
            }
            --op->n_tuned;
            return;
        }
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" rtt_status rtt_set_variant(rtt_op op, int batch, const rtt_variant* v) {
    if (!op || batch < 1 || batch > 4096) {
        set_error("invalid arguments (op=%p batch=%d)", (void*)op, batch);
        return RTT_EINVAL;
    }
    if (!v) {  // back to the default rule
        clear_variant(op, batch);
        return RTT_OK;
    }
    const int bc = v->fwd_bc;
    if (v->fwd_kernel < 1 || v->fwd_kernel > 9 || bc < 1 || bc > 64 || (bc & (bc - 1)) != 0 ||
        (bc > 32 && v->fwd_kernel < 7) ||
        v->fwd_half < 0 || v->fwd_half > 1 || v->adj_kernel < 1 || v->adj_kernel > 4) {
        set_error("invalid variant (fwd %d bc %d half %d adj %d)", v->fwd_kernel, bc, v->fwd_half,
                  v->adj_kernel);
        return RTT_EINVAL;
    }
    ApplyVariant a;
    a.fwd = (int8_t)v->fwd_kernel;
    a.fwd_bc = (int8_t)bc;
    a.fwd_half = (int8_t)v->fwd_half;
    a.adj = (int8_t)v->adj_kernel;
    if (v->fwd_order < 0 || v->fwd_order > 1) {
        set_error("invalid forward row order %d", v->fwd_order);
        return RTT_EINVAL;
    }
    a.fwd_order = (int8_t)v->fwd_order;
    if (v->fwd_cols < 0 || v->fwd_cols > 64 || v->adj_cols < 0 || v->adj_cols > 32 ||
        (v->fwd_cols & 3) || (v->adj_cols & 3)) {
        set_error("invalid column passes (forward %d, adjoint %d)", v->fwd_cols, v->adj_cols);
        return RTT_EINVAL;
    }
    a.fwd_cols = (int8_t)v->fwd_cols;
    a.adj_cols = (int8_t)v->adj_cols;
    if (v->fwd_staging < 0 || v->fwd_staging > 3) {
        set_error("invalid forward staging depth %d", v->fwd_staging);
        return RTT_EINVAL;
    }
    a.fwd_su = (int8_t)(v->fwd_staging == 0 ? 2 : v->fwd_staging);
    set_variant(op, batch, a);
    return RTT_OK;
}

extern "C" rtt_status rtt_get_variant(rtt_op op, int batch, rtt_variant* out) {
    if (!op || batch < 1 || !out) {
        set_error("invalid arguments");
        return RTT_EINVAL;
    }
    const ApplyVariant a = variant_for(op, batch);
    out->fwd_kernel = a.fwd;
    out->fwd_bc = a.fwd_bc;
    out->fwd_half = a.fwd_half;
    out->adj_kernel = a.adj;
    out->fwd_staging = a.fwd_su;
    out->fwd_order = a.fwd_order;
    out->fwd_cols = a.fwd_cols;
    out->adj_cols = a.adj_cols;
    return RTT_OK;
}

extern "C" rtt_status rtt_autotune(rtt_op op, int batch, int arm_mask, void* stream,
                                   rtt_tune_result* out) {
    if (!op || batch < 1 || batch > 4096 || !out) {
        set_error("invalid autotune arguments (op=%p batch=%d out=%p)", (void*)op, batch,
                  (void*)out);
        return RTT_EINVAL;
    }
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s != RTT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int B = batch;
    const size_t nx = (size_t)op->n_nodes * op->time.n_hats * B;
    const size_t ny = (size_t)(seg.total > 0 ? seg.total : 1) * op->time.n_frames * B;
    s = ensure_adjoint_scratch(op, B, 4);
    if (s != RTT_OK) return s;
    float *x = nullptr, *y = nullptr;
    if (cudaMalloc(&x, nx * 4) != cudaSuccess || cudaMalloc(&y, ny * 4) != cudaSuccess) {
        cudaFree(x);
        cudaFree(y);
        set_error("autotune: allocation of %zu + %zu bytes failed", nx * 4, ny * 4);
        return RTT_ENOMEM;
    }
    // timing inputs: x = 0 and y = 0 move the same bytes and issue the same
    // instructions as any data (no data-dependent branches in the kernels)
    cudaMemsetAsync(x, 0, nx * 4, st);
    cudaMemsetAsync(y, 0, ny * 4, st);

    // the rule, then candidates; a candidate is timed by installing it
    clear_variant(op, B);
    const ApplyVariant rule = variant_for(op, B);
    const bool periodic = op->frame_D > 0 && (kFracOne % op->frame_D) == 0 &&
                          (kFracOne / op->frame_D == 2 || kFracOne / op->frame_D == 4 ||
                           kFracOne / op->frame_D == 8);
    int bc_max = 1;
    while (bc_max < B && bc_max < 32) bc_max <<= 1;

    Timer tm;
    int n_cand = 0;
    cudaError_t e = cudaSuccess;
    auto time_it = [&](const ApplyVariant& v, bool adjoint) -> float {
        set_variant(op, B, v);
        ++n_cand;
        for (int w = 0; w < 1 && e == cudaSuccess; ++w)
            e = adjoint ? launch_adjoint<float>(op, y, x, B, seg, st)
                        : launch_forward<float>(op, x, y, B, seg, st);
        if (e != cudaSuccess) return 1e30f;
        cudaEventRecord(tm.a, st);
        for (int r = 0; r < kTuneReps && e == cudaSuccess; ++r)
            e = adjoint ? launch_adjoint<float>(op, y, x, B, seg, st)
                        : launch_forward<float>(op, x, y, B, seg, st);
        cudaEventRecord(tm.b, st);
        if (e != cudaSuccess) return 1e30f;
        if (cudaEventSynchronize(tm.b) != cudaSuccess) {
            e = cudaGetLastError();
            return 1e30f;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, tm.a, tm.b);
        return ms / kTuneReps;
    };

    ApplyVariant best = rule;
    // forward: staged kernel and (periodic cadences) lane-per-hat kernel, each
    // with the widest batch chunk and one or two narrower ones
    const float fwd_rule = time_it(rule, false);
    float fwd_best = fwd_rule;
    const bool x_vec = (B % 4) == 0;  // 16-byte batch records: TMA forward possible
    for (int kind = 1; kind <= 6; ++kind)
        for (int bc = bc_max; bc >= 1 && bc >= bc_max / 4; bc >>= 1)
            for (int half = 0; half <= (kind != 2 && bc < 32 ? 1 : 0); ++half) {
                ApplyVariant v = rule;
                v.fwd = (int8_t)kind;
                v.fwd_bc = (int8_t)bc;
                v.fwd_half = (int8_t)half;
                if (kind == 2 && (!periodic || bc > 8)) continue;  // lane-per-hat: <= 8 per task
                if (kind == 3 && (!x_vec || bc < 4)) continue;    // TMA: 16-byte records
                if (kind == 4 && (bc != B || (bc != 4 && bc != 8))) continue;  // one chunk
                if (kind >= 5 && (B % bc != 0 || (bc != 4 && bc != 8 && bc != 16))) continue;
                if (kind >= 5 && !periodic) continue;  // periodic specialisation
                for (int su = 1; su <= 3; ++su) {
                    // staging depth: only the staged kernel at 4 or 8 entries, full frames
                    if (su != 2 && (kind != 1 || half || (bc != 4 && bc != 8))) continue;
                    v.fwd_su = (int8_t)su;
                    const float ms = time_it(v, false);
                    if (better(ms, fwd_best)) {
                        fwd_best = ms;
                        best.fwd = v.fwd;
                        best.fwd_bc = v.fwd_bc;
                        best.fwd_half = v.fwd_half;
                        best.fwd_su = v.fwd_su;
                    }
                }
            }
    // the quad-lane forward (periodic cadences, whole 16-byte records): the
    // widest chunk of up to 64 columns dividing the batch and two narrower ones
    if (periodic && x_vec) {
        int qbc = 64;
        while (B % qbc != 0) qbc >>= 1;
        for (int kind = 7; kind <= 9; ++kind)
            for (int bc = qbc; bc >= 4 && bc >= qbc / 4; bc >>= 1)
                for (int half = 0; half <= 1; ++half) {
                    ApplyVariant v = rule;
                    v.fwd = (int8_t)kind;
                    v.fwd_bc = (int8_t)bc;
                    v.fwd_half = (int8_t)half;
                    v.fwd_su = 2;
                    const float ms = time_it(v, false);
                    if (better(ms, fwd_best)) {
                        fwd_best = ms;
                        best.fwd = v.fwd;
                        best.fwd_bc = v.fwd_bc;
                        best.fwd_half = v.fwd_half;
                        best.fwd_su = v.fwd_su;
                    }
                }
    }
    // the same kernels for 1- or 2-column batches (16-byte units of 4 / B frames)
    if (periodic && B <= 2)
        for (int kind = 7; kind <= 8; ++kind)
            for (int half = 0; half <= 1; ++half) {
                ApplyVariant v = rule;
                v.fwd = (int8_t)kind;
                v.fwd_bc = (int8_t)B;
                v.fwd_half = (int8_t)half;
                v.fwd_su = 2;
                const float ms = time_it(v, false);
                if (better(ms, fwd_best)) {
                    fwd_best = ms;
                    best.fwd = v.fwd;
                    best.fwd_bc = v.fwd_bc;
                    best.fwd_half = v.fwd_half;
                    best.fwd_su = v.fwd_su;
                }
            }
    // forward task rows in source-cell order, for the chosen kernel
    {
        ApplyVariant v = best;
        v.fwd_order = 1;
        const float ms = time_it(v, false);
        if (better(ms, fwd_best)) {
            fwd_best = ms;
            best.fwd_order = 1;
        }
    }
    // forward column passes of 8 columns (large batches of the periodic forward)
    if ((best.fwd == 5 || best.fwd == 6) && B > 8 && B % 8 == 0) {
        ApplyVariant v = best;
        v.fwd_cols = 8;
        const float ms = time_it(v, false);
        if (better(ms, fwd_best)) {
            fwd_best = ms;
            best.fwd_cols = 8;
        }
    }
    // adjoint: the per-lane staged kernel and the TMA kernels the call allows
    const float adj_rule = time_it(rule, true);
    float adj_best = adj_rule;
    const int adj_max = adjoint_best_kind(op, B);
    for (int k = 1; k <= adj_max; ++k) {
        ApplyVariant v = best;
        v.adj = (int8_t)k;
        const float ms = time_it(v, true);
        if (better(ms, adj_best)) {
            adj_best = ms;
            best.adj = v.adj;
        }
    }
    // adjoint passes of 8, 16 or 32 columns (large batches; 32 where the
    // default is 64-column passes)
    for (int pc = 8; pc <= 32 && B > pc; pc *= 2) {
        ApplyVariant v = best;
        v.adj_cols = (int8_t)pc;
        const float ms = time_it(v, true);
        if (better(ms, adj_best)) {
            adj_best = ms;
            best.adj_cols = (int8_t)pc;
        }
    }
    cudaFree(x);
    cudaFree(y);
    if (e != cudaSuccess) {
        clear_variant(op, B);
        set_error("autotune launch failed: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    set_variant(op, B, best);
    out->batch = B;
    out->fwd_kernel = best.fwd;
    out->fwd_bc = best.fwd_bc;
    out->fwd_staging = best.fwd_su;
    out->fwd_frames_per_lane =
        best.fwd == 2 ? (int32_t)(kFracOne / op->frame_D)
                      : (best.fwd_bc >= 32 ? 1 : (32 / best.fwd_bc) / (best.fwd_half ? 2 : 1));
    out->adj_kernel = best.adj;
    out->fwd_order = best.fwd_order;
    out->fwd_cols = best.fwd_cols;
    out->adj_cols = best.adj_cols;
    out->fwd_ms = fwd_best;
    out->adj_ms = adj_best;
    out->fwd_ms_rule = fwd_rule;
    out->adj_ms_rule = adj_rule;
    out->candidates = n_cand;
    return RTT_OK;
}
