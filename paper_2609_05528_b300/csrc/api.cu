// C ABI entry points: operator construction (table preparation on the
// device), queries, and the forward / adjoint applies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <cub/cub.cuh>
#include <string>
#include <vector>

#include "rtt_internal.cuh"

namespace rtt {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}


#define RTT_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t _e = (call);                                                        \
        if (_e != cudaSuccess) {                                                        \
            set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, \
                      __LINE__);                                                        \
            return _e == cudaErrorMemoryAllocation ? RTT_ENOMEM : RTT_ECUDA;            \
        }                                                                               \
    } while (0)

// --------------------------------------------------------------------------
// Table preparation kernels (K8)
// --------------------------------------------------------------------------
__global__ void make_row_keys(int64_t n, const int8_t* order, const int32_t* pixel,
                              unsigned long long* key, int32_t* idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = ((unsigned long long)(uint8_t)order[i] << 32) | (unsigned long long)(uint32_t)pixel[i];
    idx[i] = (int32_t)i;
}

__global__ void row_flags(int64_t n, const unsigned long long* key, int32_t* flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// rows[i] = inclusive scan - 1; row_ptr[row] = first ray; row order histogram
__global__ void row_index(int64_t n, const unsigned long long* key, const int32_t* flag,
                          const int32_t* incl, int32_t* ray_row, int32_t* row_ptr,
                          int32_t* row_order, int32_t* row_pixel, unsigned int* order_count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t row = incl[i] - 1;
    ray_row[i] = row;
    if (flag[i]) {
        row_ptr[row] = (int32_t)i;
        const int ord = (int)(key[i] >> 32);
        row_order[row] = ord;
        row_pixel[row] = (int32_t)(uint32_t)(key[i] & 0xffffffffull);
        atomicAdd(&order_count[ord], 1u);  // integer counts: order independent
    }
}

// FP32 corner weights from the FP64 ones (rounded to nearest), optionally
// rounded on to BF16 (nearest even) with the packed BF16 copy
__global__ void set_weights(int64_t n, const double* __restrict__ W64, int bf16, float4* W, uint2* W16) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float c[4];
    for (int q = 0; q < 4; ++q) {
        c[q] = (float)W64[4 * i + q];
        if (bf16) c[q] = __bfloat162float(__float2bfloat16_rn(c[q]));
    }
    W[i] = make_float4(c[0], c[1], c[2], c[3]);
    if (bf16)
        W16[i] = make_uint2((__float_as_uint(c[1]) & 0xffff0000u) | (__float_as_uint(c[0]) >> 16),
                            (__float_as_uint(c[3]) & 0xffff0000u) | (__float_as_uint(c[2]) >> 16));
}

// out[i] = in[i] - base (row pointers and row indices of a row shard)
__global__ void rebase_rows(int64_t n, const int32_t* in, int32_t base, int32_t* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i] - base;
}

struct PrepArgs {
    int64_t n;
    const int32_t* perm;
    const double* r;
    const double* phi;
    const double* delay;
    const double* weight;
    const double* thr;
    int n_r, n_phi;
    double log_rin, log_rout;
    double t0, t_end, hat_step;
    double scale;
    int32_t* node00;
    int32_t* node01;
    float4* W;
    double* W64;
    int32_t* K0;
    int32_t* F0;
    double* F64;
    double* r_s;
    double* phi_s;
    double* delay_s;
    double* weight_s;
    double* thr_s;
};

// Per sorted ray: bilinear stencil in (log r, phi) and integer hat offset,
// all derived in FP64 (Eq. 2 interpolation of the nodal history).
__global__ void prep_rays(const PrepArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int32_t o = a.perm[i];
    const double r = a.r[o], phi = a.phi[o], dl = a.delay[o], w = a.weight[o];
    double rho = (log(r) - a.log_rin) / (a.log_rout - a.log_rin) * (double)(a.n_r - 1);
    int i0 = (int)floor(rho);
    i0 = max(0, min(i0, a.n_r - 2));
    const double fr = rho - (double)i0;
    const double twopi = 6.283185307179586476925286766559;
    double ph = phi / twopi * (double)a.n_phi;
    ph = fmod(ph, (double)a.n_phi);
    if (ph < 0.0) ph += (double)a.n_phi;
    int j0 = (int)floor(ph);
    if (j0 >= a.n_phi) j0 = a.n_phi - 1;
    const double fp = ph - (double)j0;
    const int j1 = (j0 + 1) % a.n_phi;
    a.node00[i] = i0 * a.n_phi + j0;
    a.node01[i] = i0 * a.n_phi + j1;
    const double sw = a.scale * w;
    const double c00 = sw * (1.0 - fr) * (1.0 - fp);
    const double c10 = sw * fr * (1.0 - fp);
    const double c01 = sw * (1.0 - fr) * fp;
    const double c11 = sw * fr * fp;
    a.W64[4 * i + 0] = c00;
    a.W64[4 * i + 1] = c10;
    a.W64[4 * i + 2] = c01;
    a.W64[4 * i + 3] = c11;
    a.W[i] = make_float4((float)c00, (float)c10, (float)c01, (float)c11);
    // hat coordinate u(f) = (t_end - t_o(f) + Delta) / hat_step = u0 - f delta
    const double u0 = (a.t_end - a.t0 + dl) / a.hat_step;
    const double k0 = floor(u0);
    const double frac = u0 - k0;
    double fq = floor(frac * (double)kFracOne);
    if (fq > (double)kFracMask) fq = (double)kFracMask;
    if (fq < 0.0) fq = 0.0;
    a.K0[i] = (int32_t)k0;
    a.F0[i] = (int32_t)fq;
    a.F64[i] = frac;
    a.r_s[i] = r;
    a.phi_s[i] = phi;
    a.delay_s[i] = dl;
    a.weight_s[i] = w;
    a.thr_s[i] = a.thr[o];
}

// Per direct row: sum_e w_e (FP64, sequential over the row's rays); squared.
__global__ void row_weight_sq(int64_t n_rows, const int32_t* row_ptr, const double* w,
                              double* out) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n_rows) return;
    double s = 0.0;
    for (int e = row_ptr[row]; e < row_ptr[row + 1]; ++e) s += w[e];
    out[row] = s * s;
}

static bool dyadic_delta(double cadence, double hat_step, int64_t* D) {
    const double d = cadence / hat_step;
    const double q = d * (double)kFracOne;
    if (!(q >= 1.0) || q != floor(q) || d > 1.0) return false;
    *D = (int64_t)q;
    return true;
}

static rtt_status check_grids(const rtt_source_grid* g, const rtt_time_grid* t) {
    if (g->n_r < 2 || g->n_phi < 2 || !(g->r_in > 0.0) || !(g->r_out > g->r_in) ||
        (int64_t)g->n_r * g->n_phi > (1 << 28)) {
        set_error("invalid source grid (n_r=%d n_phi=%d r_in=%g r_out=%g)", g->n_r, g->n_phi,
                  g->r_in, g->r_out);
        return RTT_EINVAL;
    }
    if (t->n_frames < 1 || t->n_hats < 1 || !(t->cadence > 0.0) || !(t->hat_step > 0.0) ||
        !std::isfinite(t->t0) || !std::isfinite(t->t_end)) {
        set_error("invalid time grid");
        return RTT_EINVAL;
    }
    int64_t D;
    if (!dyadic_delta(t->cadence, t->hat_step, &D)) {
        set_error("cadence/hat_step = %g must be a multiple of 2^-24 in (0, 1]",
                  t->cadence / t->hat_step);
        return RTT_EINVAL;
    }
    return RTT_OK;
}

template <typename T>
static rtt_status alloc(T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T) + 16);
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu) failed: %s", n * sizeof(T), cudaGetErrorString(e));
        *p = nullptr;
        return RTT_ENOMEM;
    }
    return RTT_OK;
}

static void free_op(rtt_op_s* op) {
    if (!op) return;
    void* ps[] = {op->row_ptr, op->ray_row, op->node00, op->node01, op->W,     op->W64,
                  op->K0,      op->F0,      op->F64,    op->r,      op->delay, op->weight,
                  op->thr,     op->row_order, op->c_row, op->c_col, op->c_K0, op->c_F0, op->c_fb, op->c_r0,
                  op->c_W,     op->c_W64,   op->c_F64, op->seg_ray, op->seg_col, op->seg_ncol,
                  op->seg_rec, op->gslot,   op->adj_ctr, op->cpart, op->row_sched,
                  op->W16,     op->c_W16,   op->cell_ptr, op->ray_rec,
                  op->dev_status, op->rscratch, op->row_pixel, op->mix.grp_ptr,
                  op->mix.grp_rows, op->mix.row_grp, op->mix.inv32, op->mix.inv64,
                  op->mix.part, op->phi};
    for (void* p : ps)
        if (p) cudaFree(p);
    delete op;
}

static int blocks(int64_t n, int t = 256) { return (int)((n + t - 1) / t); }

// Scoped device buffers for the build (freed on every exit path).
struct Scratch {
    std::vector<void*> ptrs;
    ~Scratch() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    rtt_status get(T** p, size_t n) {
        RTT_TRY(alloc(p, n));
        ptrs.push_back(*p);
        return RTT_OK;
    }
};

// Rows [lo, hi) of shard `index` of `count` over R rows: contiguous blocks of
// the (order, pixel)-sorted rows, sizes differing by at most one.
static void shard_rows(int64_t R, int index, int count, int64_t* lo, int64_t* hi) {
    *lo = R * (int64_t)index / count;
    *hi = R * (int64_t)(index + 1) / count;
}

// the forward's per-ray record: (K0, F0, node00, node01) as int bits, then the
// corner weights W (all = false: the weights only, after a precision change)
__global__ void pack_ray_rec(int64_t n, const int32_t* __restrict__ K0, const int32_t* __restrict__ F0,
                             const int32_t* __restrict__ n00, const int32_t* __restrict__ n01,
                             const float4* __restrict__ W, bool all, float4* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    if (all)
        out[2 * e] = make_float4(__int_as_float(K0[e]), __int_as_float(F0[e]), __int_as_float(n00[e]),
                                 __int_as_float(n01[e]));
    out[2 * e + 1] = W[e];
}

static rtt_status build_impl(const rtt_geometry* geom, const rtt_source_grid* grid,
                             const rtt_time_grid* time, const rtt_ray_table* tab,
                             const rtt_options* opt, const rtt_shard* shard, cudaStream_t st,
                             rtt_op_s* op) {
    const int64_t E = tab->n_rays;
    // ---- host validation pass (also yields per-order delay ranges) ----
    for (int n = 0; n < 3; ++n) {
        op->dmin[n] = INFINITY;
        op->dmax[n] = -INFINITY;
    }
    int64_t n_direct = 0;
    for (int64_t i = 0; i < E; ++i) {
        const int o = tab->order[i];
        const double r = tab->r[i], ph = tab->phi[i], d = tab->delay[i], w = tab->weight[i],
                     th = tab->throughput[i];
        if (o < 0 || o > 2 || tab->pixel[i] < 0) {
            set_error("ray %lld: order %d / pixel %d out of range", (long long)i, o, tab->pixel[i]);
            return RTT_EINVAL;
        }
        if (!std::isfinite(r) || !std::isfinite(ph) || !std::isfinite(d) || !std::isfinite(w) ||
            !std::isfinite(th) || std::fabs(ph) > 1e6 || std::fabs(d) > 1e6) {
            set_error("ray %lld: non-finite or out-of-range value", (long long)i);
            return RTT_EINVAL;
        }
        if (r < grid->r_in || r > grid->r_out) {
            set_error("ray %lld: r = %.17g outside [r_in, r_out]", (long long)i, r);
            return RTT_EINVAL;
        }
        const double u0 = (time->t_end - time->t0 + d) / time->hat_step;
        if (std::fabs(u0) > 1048576.0) {  // |u0| <= 2^20 hat steps
            set_error("ray %lld: hat offset out of range", (long long)i);
            return RTT_EINVAL;
        }
        op->dmin[o] = std::fmin(op->dmin[o], d);
        op->dmax[o] = std::fmax(op->dmax[o], d);
        n_direct += (o == 0);
    }
    if (n_direct == 0) {
        set_error("the table has no direct (order 0) ray");
        return RTT_EINVAL;
    }
    for (int n = 0; n < 3; ++n)
        if (!(op->dmin[n] <= op->dmax[n])) op->dmin[n] = op->dmax[n] = NAN;
    op->geom = *geom;
    op->grid = *grid;
    op->time = *time;
    op->opt = *opt;
    op->n_rays = E;
    op->n_nodes = grid->n_r * grid->n_phi;
    dyadic_delta(time->cadence, time->hat_step, &op->frame_D);
    op->delta = time->cadence / time->hat_step;

    Scratch sc;
    int8_t* d_order;
    int32_t* d_pixel;
    double *d_r, *d_phi, *d_delay, *d_w, *d_thr;
    RTT_TRY(sc.get(&d_order, E));
    RTT_TRY(sc.get(&d_pixel, E));
    RTT_TRY(sc.get(&d_r, E));
    RTT_TRY(sc.get(&d_phi, E));
    RTT_TRY(sc.get(&d_delay, E));
    RTT_TRY(sc.get(&d_w, E));
    RTT_TRY(sc.get(&d_thr, E));
    RTT_CUDA(cudaMemcpyAsync(d_order, tab->order, E, cudaMemcpyHostToDevice, st));
    RTT_CUDA(cudaMemcpyAsync(d_pixel, tab->pixel, E * 4, cudaMemcpyHostToDevice, st));
    RTT_CUDA(cudaMemcpyAsync(d_r, tab->r, E * 8, cudaMemcpyHostToDevice, st));
    RTT_CUDA(cudaMemcpyAsync(d_phi, tab->phi, E * 8, cudaMemcpyHostToDevice, st));
    RTT_CUDA(cudaMemcpyAsync(d_delay, tab->delay, E * 8, cudaMemcpyHostToDevice, st));
    RTT_CUDA(cudaMemcpyAsync(d_w, tab->weight, E * 8, cudaMemcpyHostToDevice, st));
    RTT_CUDA(cudaMemcpyAsync(d_thr, tab->throughput, E * 8, cudaMemcpyHostToDevice, st));

    // ---- row CSR: stable device radix sort of rays by (order, pixel) ----
    unsigned long long *k_in, *k_out;
    int32_t *v_in, *perm, *flag, *incl;
    unsigned int* ocount;
    RTT_TRY(sc.get(&k_in, E));
    RTT_TRY(sc.get(&k_out, E));
    RTT_TRY(sc.get(&v_in, E));
    RTT_TRY(sc.get(&perm, E));
    RTT_TRY(sc.get(&flag, E));
    RTT_TRY(sc.get(&incl, E));
    RTT_TRY(sc.get(&ocount, 4));
    RTT_CUDA(cudaMemsetAsync(ocount, 0, 16, st));
    make_row_keys<<<blocks(E), 256, 0, st>>>(E, d_order, d_pixel, k_in, v_in);
    RTT_CUDA(cudaGetLastError());
    size_t tmp_bytes = 0;
    RTT_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, k_in, k_out, v_in, perm, E, 0, 34,
                                             st));
    size_t tmp2 = 0;
    RTT_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tmp2, flag, incl, E, st));
    tmp_bytes = tmp_bytes > tmp2 ? tmp_bytes : tmp2;
    void* d_tmp;
    RTT_TRY(sc.get((unsigned char**)&d_tmp, tmp_bytes));

    size_t tb = tmp_bytes;
    RTT_CUDA(cub::DeviceRadixSort::SortPairs(d_tmp, tb, k_in, k_out, v_in, perm, E, 0, 34, st));
    row_flags<<<blocks(E), 256, 0, st>>>(E, k_out, flag);
    RTT_CUDA(cudaGetLastError());
    tb = tmp_bytes;
    RTT_CUDA(cub::DeviceScan::InclusiveSum(d_tmp, tb, flag, incl, E, st));
    int32_t n_rows_i = 0;
    RTT_CUDA(cudaMemcpyAsync(&n_rows_i, incl + (E - 1), 4, cudaMemcpyDeviceToHost, st));
    RTT_CUDA(cudaStreamSynchronize(st));
    const int64_t R = n_rows_i;
    op->n_rows = R;
    RTT_TRY(alloc(&op->row_ptr, R + 1));
    RTT_TRY(alloc(&op->ray_row, E));
    RTT_TRY(alloc(&op->row_order, R));
    RTT_TRY(alloc(&op->row_pixel, R));
    row_index<<<blocks(E), 256, 0, st>>>(E, k_out, flag, incl, op->ray_row, op->row_ptr,
                                         op->row_order, op->row_pixel, ocount);
    RTT_CUDA(cudaGetLastError());
    const int32_t E32 = (int32_t)E;
    RTT_CUDA(cudaMemcpyAsync(op->row_ptr + R, &E32, 4, cudaMemcpyHostToDevice, st));
    unsigned int hcount[4];
    RTT_CUDA(cudaMemcpyAsync(hcount, ocount, 16, cudaMemcpyDeviceToHost, st));
    RTT_CUDA(cudaStreamSynchronize(st));
    op->row_begin[0] = 0;
    for (int n = 0; n < 3; ++n) op->row_begin[n + 1] = op->row_begin[n] + hcount[n];

    // ---- s_ref (Eq. 17, j_ref = 1 evaluated directly) ----
    RTT_TRY(alloc(&op->r, E));
    RTT_TRY(alloc(&op->phi, E));
    RTT_TRY(alloc(&op->delay, E));
    RTT_TRY(alloc(&op->weight, E));
    RTT_TRY(alloc(&op->thr, E));
    // first prep pass with scale = 1 yields the sorted raw weights for s_ref
    RTT_TRY(alloc(&op->node00, E));
    RTT_TRY(alloc(&op->node01, E));
    RTT_TRY(alloc(&op->W, E));
    RTT_TRY(alloc(&op->W64, 4 * E));
    RTT_TRY(alloc(&op->K0, E));
    RTT_TRY(alloc(&op->F0, E));
    RTT_TRY(alloc(&op->F64, E));
    PrepArgs pa{};
    pa.n = E;
    pa.perm = perm;
    pa.r = d_r;
    pa.phi = d_phi;
    pa.delay = d_delay;
    pa.weight = d_w;
    pa.thr = d_thr;
    pa.n_r = grid->n_r;
    pa.n_phi = grid->n_phi;
    pa.log_rin = log(grid->r_in);
    pa.log_rout = log(grid->r_out);
    pa.t0 = time->t0;
    pa.t_end = time->t_end;
    pa.hat_step = time->hat_step;
    pa.scale = 1.0;
    pa.node00 = op->node00;
    pa.node01 = op->node01;
    pa.W = op->W;
    pa.W64 = op->W64;
    pa.K0 = op->K0;
    pa.F0 = op->F0;
    pa.F64 = op->F64;
    pa.r_s = op->r;
    pa.phi_s = op->phi;
    pa.delay_s = op->delay;
    pa.weight_s = op->weight;
    pa.thr_s = op->thr;
    prep_rays<<<blocks(E), 256, 0, st>>>(pa);
    RTT_CUDA(cudaGetLastError());
    const int64_t R0 = op->row_begin[1];
    double *rsq, *rsum;
    RTT_TRY(sc.get(&rsq, R0));
    RTT_TRY(sc.get(&rsum, 1));
    row_weight_sq<<<blocks(R0), 256, 0, st>>>(R0, op->row_ptr, op->weight, rsq);
    RTT_CUDA(cudaGetLastError());
    size_t tmp5 = 0;
    RTT_CUDA(cub::DeviceReduce::Sum(nullptr, tmp5, rsq, rsum, R0, st));
    if (tmp5 > tmp_bytes) {
        set_error("internal: reduce scratch too small");
        return RTT_ECUDA;
    }
    tb = tmp_bytes;
    RTT_CUDA(cub::DeviceReduce::Sum(d_tmp, tb, rsq, rsum, R0, st));
    double hsum = 0.0;
    RTT_CUDA(cudaMemcpyAsync(&hsum, rsum, 8, cudaMemcpyDeviceToHost, st));
    RTT_CUDA(cudaStreamSynchronize(st));
    op->s_ref = sqrt(hsum / (double)R0);
    if (!(op->s_ref > 0.0)) {
        set_error("s_ref = %g: direct weights are zero", op->s_ref);
        return RTT_EINVAL;
    }
    op->scale = opt->snr0 / op->s_ref;
    op->total_rows = R;
    for (int n = 0; n < 4; ++n) op->total_row_begin[n] = op->row_begin[n];
    op->shard_index = 0;
    op->shard_count = 1;
    op->shard_row_begin = 0;
    // ---- row shard: keep rows [lo, hi) of the sorted row list and their rays,
    // which are the sorted rays [row_ptr[lo], row_ptr[hi]); s_ref and the
    // scale above are those of the whole table ----
    if (shard && shard->count > 1) {
        int64_t lo = 0, hi = 0;
        shard_rows(R, shard->index, shard->count, &lo, &hi);
        if (hi <= lo) {
            set_error("shard %d of %d has no rows (%lld rows in the table)", shard->index,
                      shard->count, (long long)R);
            return RTT_EINVAL;
        }
        int32_t eb[2];
        RTT_CUDA(cudaMemcpyAsync(&eb[0], op->row_ptr + lo, 4, cudaMemcpyDeviceToHost, st));
        RTT_CUDA(cudaMemcpyAsync(&eb[1], op->row_ptr + hi, 4, cudaMemcpyDeviceToHost, st));
        RTT_CUDA(cudaStreamSynchronize(st));
        const int64_t Rs = hi - lo, e_lo = eb[0], Es = (int64_t)eb[1] - eb[0];
        int32_t *rp, *rr, *ro, *rpx;
        RTT_TRY(alloc(&rp, Rs + 1));
        RTT_TRY(alloc(&rr, Es));
        RTT_TRY(alloc(&ro, Rs));
        RTT_TRY(alloc(&rpx, Rs));
        rebase_rows<<<blocks(Rs + 1), 256, 0, st>>>(Rs + 1, op->row_ptr + lo, (int32_t)e_lo, rp);
        rebase_rows<<<blocks(Es), 256, 0, st>>>(Es, op->ray_row + e_lo, (int32_t)lo, rr);
        RTT_CUDA(cudaGetLastError());
        RTT_CUDA(cudaMemcpyAsync(ro, op->row_order + lo, Rs * 4, cudaMemcpyDeviceToDevice, st));
        RTT_CUDA(cudaMemcpyAsync(rpx, op->row_pixel + lo, Rs * 4, cudaMemcpyDeviceToDevice, st));
        RTT_CUDA(cudaStreamSynchronize(st));
        void* old_arrays[] = {op->row_ptr, op->ray_row, op->row_order, op->row_pixel, op->node00,
                              op->node01,  op->W,       op->W64,       op->K0,         op->F0,
                              op->F64,     op->r,       op->phi,       op->delay,      op->weight,
                              op->thr};
        for (void* q : old_arrays) cudaFree(q);
        op->row_ptr = rp;
        op->ray_row = rr;
        op->row_order = ro;
        op->row_pixel = rpx;
        op->node00 = op->node01 = op->K0 = op->F0 = nullptr;
        op->W = nullptr;
        op->W64 = op->F64 = op->r = op->phi = op->delay = op->weight = op->thr = nullptr;
        RTT_TRY(alloc(&op->r, Es));
        RTT_TRY(alloc(&op->phi, Es));
        RTT_TRY(alloc(&op->delay, Es));
        RTT_TRY(alloc(&op->weight, Es));
        RTT_TRY(alloc(&op->thr, Es));
        RTT_TRY(alloc(&op->node00, Es));
        RTT_TRY(alloc(&op->node01, Es));
        RTT_TRY(alloc(&op->W, Es));
        RTT_TRY(alloc(&op->W64, 4 * Es));
        RTT_TRY(alloc(&op->K0, Es));
        RTT_TRY(alloc(&op->F0, Es));
        RTT_TRY(alloc(&op->F64, Es));
        // order blocks of the shard: the global blocks clipped to [lo, hi)
        for (int n = 0; n < 4; ++n) {
            const int64_t b = op->row_begin[n] - lo;
            op->row_begin[n] = b < 0 ? 0 : (b > Rs ? Rs : b);
        }
        op->n_rows = Rs;
        op->n_rays = Es;
        op->shard_index = shard->index;
        op->shard_count = shard->count;
        op->shard_row_begin = lo;
        pa.n = Es;
        pa.perm = perm + e_lo;
        pa.node00 = op->node00;
        pa.node01 = op->node01;
        pa.W = op->W;
        pa.W64 = op->W64;
        pa.K0 = op->K0;
        pa.F0 = op->F0;
        pa.F64 = op->F64;
        pa.r_s = op->r;
        pa.phi_s = op->phi;
        pa.delay_s = op->delay;
        pa.weight_s = op->weight;
        pa.thr_s = op->thr;
    }
    // second pass with the whitening scale folded into the corner weights
    pa.scale = op->scale;
    prep_rays<<<blocks(pa.n), 256, 0, st>>>(pa);
    RTT_CUDA(cudaGetLastError());

    // ---- the forward's source-cell row order: within each order, rows by the
    // Morton index of their first ray's cell (i0, j0) (ties by row) ----
    {
        const int64_t R = op->n_rows, E = op->n_rays;
        std::vector<int32_t> rp(R + 1), n00(E);
        RTT_CUDA(cudaMemcpyAsync(rp.data(), op->row_ptr, (R + 1) * 4, cudaMemcpyDeviceToHost, st));
        RTT_CUDA(cudaMemcpyAsync(n00.data(), op->node00, E * 4, cudaMemcpyDeviceToHost, st));
        RTT_CUDA(cudaStreamSynchronize(st));
        auto morton = [](uint32_t i, uint32_t j) {
            uint64_t m = 0;
            for (int b = 0; b < 16; ++b)
                m |= (uint64_t)((i >> b) & 1u) << (2 * b + 1) | (uint64_t)((j >> b) & 1u) << (2 * b);
            return m;
        };
        std::vector<uint64_t> key(R);
        for (int64_t r = 0; r < R; ++r) {
            const int32_t c = n00[rp[r]];
            key[r] = morton((uint32_t)(c / grid->n_phi), (uint32_t)(c % grid->n_phi));
        }
        std::vector<int32_t> sched(R);
        for (int64_t r = 0; r < R; ++r) sched[r] = (int32_t)r;
        for (int n = 0; n < 3; ++n)
            std::stable_sort(sched.begin() + op->row_begin[n], sched.begin() + op->row_begin[n + 1],
                             [&](int32_t a, int32_t b) { return key[a] < key[b]; });
        RTT_TRY(alloc(&op->row_sched, R));
        RTT_CUDA(cudaMemcpy(op->row_sched, sched.data(), R * 4, cudaMemcpyHostToDevice));
    }
    // the forward's per-ray fields packed into one 32-byte record (two loads
    // from one sector per ray instead of five from five arrays)
    RTT_TRY(alloc(&op->ray_rec, 2 * op->n_rays));
    if (op->n_rays > 0) {
        pack_ray_rec<<<blocks(op->n_rays), 256, 0, st>>>(op->n_rays, op->K0, op->F0, op->node00,
                                                         op->node01, op->W, true, op->ray_rec);
        RTT_CUDA(cudaGetLastError());
    }
    RTT_TRY(alloc(&op->dev_status, 1));
    RTT_CUDA(cudaMemsetAsync(op->dev_status, 0, sizeof(int), st));
    // ---- the adjoint's cell structures (rays by source cell, strip segments) ----
    RTT_TRY(build_cells(op, st));
    return RTT_OK;
}

rtt_status make_seg(const rtt_op_s* op, int mask, ArmSeg* s) {
    if (mask < 1 || mask > 7) {
        set_error("arm_mask %d not in 1..7", mask);
        return RTT_EINVAL;
    }
    s->n = 0;
    s->total = 0;
    s->mask = mask;
    for (int n = 0; n < 3; ++n) {
        if (!(mask & (1 << n))) continue;
        const int64_t len = op->row_begin[n + 1] - op->row_begin[n];
        if (len == 0) continue;
        s->begin[s->n] = (int32_t)op->row_begin[n];
        s->len[s->n] = (int32_t)len;
        s->out_off[s->n] = s->total;
        s->total += (int32_t)len;
        s->n += 1;
    }
    for (int i = s->n; i < 3; ++i) s->begin[i] = s->len[i] = s->out_off[i] = 0;
    return RTT_OK;
}

// Grow-only adjoint scratch owned by the operator.  Growing frees the old
// buffer after synchronising the device, so calls that need more scratch
// than any earlier call are synchronous once.

// r = y - d, elementwise (FP32, one rounding)
__global__ void residual_kernel(const float* __restrict__ y, const float* __restrict__ d,
                                float* __restrict__ r, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        r[i] = y[i] - d[i];
}

template <typename T>
static rtt_status apply_common(rtt_op op, const T* in, T* out, int batch, int mask, void* stream,
                               bool adjoint) {
    if (!op || batch < 1) {
        set_error("invalid argument (op=%p batch=%d)", (void*)op, batch);
        return RTT_EINVAL;
    }
    ArmSeg seg;
    RTT_TRY(make_seg(op, mask, &seg));
    // data-side pointers may be null only when the arm selects no rows
    const bool need_in = adjoint ? seg.total > 0 : true;
    const bool need_out = adjoint ? true : seg.total > 0;
    if ((need_in && !in) || (need_out && !out)) {
        set_error("null buffer (in=%p out=%p, arm rows %d)", (const void*)in, (void*)out,
                  seg.total);
        return RTT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (adjoint) {
        RTT_TRY(ensure_adjoint_scratch(op, batch, (int)sizeof(T)));
        e = launch_adjoint<T>(op, in, out, batch, seg, st);
    } else {
        e = launch_forward<T>(op, in, out, batch, seg, st);
    }
    if (e != cudaSuccess) {
        set_error("apply launch failed: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    return RTT_OK;
}

}  // namespace rtt

using namespace rtt;

extern "C" {

const char* rtt_error_string(rtt_status s) {
    switch (s) {
        case RTT_OK: return "ok";
        case RTT_EINVAL: return "invalid argument";
        case RTT_ENOMEM: return "out of memory";
        case RTT_ECUDA: return "CUDA error";
        case RTT_ETIMEOUT: return "device wait timed out";
        case RTT_ENOTCONVERGED: return "iteration did not converge";
        case RTT_ESTATE: return "invalid state";
        case RTT_EDEVICE: return "device-side check failed";
    }
    return "unknown status";
}

const char* rtt_last_error(void) { return g_last_error.c_str(); }

int rtt_abi_version(void) { return RTT_ABI_VERSION; }

rtt_status rtt_build_operator_shard(const rtt_geometry* geom, const rtt_source_grid* grid,
                                    const rtt_time_grid* time, const rtt_ray_table* table,
                                    const rtt_options* opt, const rtt_shard* shard, void* stream,
                                    rtt_op* out) {
    if (!geom || !grid || !time || !table || !opt || !out) {
        set_error("null argument");
        return RTT_EINVAL;
    }
    *out = nullptr;
    if (shard && (shard->count < 1 || shard->index < 0 || shard->index >= shard->count)) {
        set_error("shard index %d of %d invalid", shard->index, shard->count);
        return RTT_EINVAL;
    }
    if (table->n_rays < 1 || table->n_rays > (1ll << 29) || !table->order || !table->pixel ||
        !table->r || !table->phi || !table->delay || !table->weight || !table->throughput) {
        set_error("invalid ray table (n_rays=%lld)", (long long)table->n_rays);
        return RTT_EINVAL;
    }
    if (!(opt->snr0 > 0.0) || !(opt->rho > 0.0)) {
        set_error("snr0 and rho must be positive");
        return RTT_EINVAL;
    }
    if (!(std::fabs(geom->spin) < 1.0)) {
        set_error("spin must satisfy |a| < 1");
        return RTT_EINVAL;
    }
    RTT_TRY(check_grids(grid, time));
    rtt_op_s* op = new (std::nothrow) rtt_op_s();
    if (!op) {
        set_error("host allocation failed");
        return RTT_ENOMEM;
    }
    rtt_status s = build_impl(geom, grid, time, table, opt, shard, (cudaStream_t)stream, op);
    if (s != RTT_OK) {
        free_op(op);
        return s;
    }
    *out = op;
    return RTT_OK;
}

rtt_status rtt_build_operator(const rtt_geometry* geom, const rtt_source_grid* grid,
                              const rtt_time_grid* time, const rtt_ray_table* table,
                              const rtt_options* opt, void* stream, rtt_op* out) {
    return rtt_build_operator_shard(geom, grid, time, table, opt, nullptr, stream, out);
}

rtt_status rtt_set_weight_precision(rtt_op op, int precision, void* stream) {
    if (!op || (precision != RTT_WEIGHTS_FP32 && precision != RTT_WEIGHTS_BF16)) {
        set_error("invalid weight precision %d", precision);
        return RTT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t E = op->n_rays;
    const bool bf16 = precision == RTT_WEIGHTS_BF16;
    if (bf16 && !op->W16) {
        RTT_TRY(alloc(&op->W16, E));
        RTT_TRY(alloc(&op->c_W16, E));
    }
    const int nb = (int)((E + 255) / 256);
    set_weights<<<nb, 256, 0, st>>>(E, op->W64, bf16, op->W, op->W16);
    set_weights<<<nb, 256, 0, st>>>(E, op->c_W64, bf16, op->c_W, op->c_W16);
    if (op->ray_rec)  // the record's copy of the (re-rounded) weights
        pack_ray_rec<<<nb, 256, 0, st>>>(E, op->K0, op->F0, op->node00, op->node01, op->W, false,
                                         op->ray_rec);
    RTT_CUDA(cudaGetLastError());
    RTT_CUDA(cudaStreamSynchronize(st));
    if (!bf16 && op->W16) {
        cudaFree(op->W16);
        cudaFree(op->c_W16);
        op->W16 = op->c_W16 = nullptr;
    }
    op->weight_precision = precision;
    return RTT_OK;
}

rtt_status rtt_shard_rows(int64_t n_rows, const rtt_shard* shard, int64_t* begin_out,
                          int64_t* end_out) {
    if (!shard || !begin_out || !end_out || n_rows < 0 || shard->count < 1 ||
        shard->index < 0 || shard->index >= shard->count) {
        set_error("invalid shard (n_rows=%lld)", (long long)n_rows);
        return RTT_EINVAL;
    }
    shard_rows(n_rows, shard->index, shard->count, begin_out, end_out);
    return RTT_OK;
}

rtt_status rtt_op_query(rtt_op op, rtt_op_info* o) {
    if (!op || !o) {
        set_error("null argument");
        return RTT_EINVAL;
    }
    o->n_rays = op->n_rays;
    o->n_rows = op->n_rows;
    for (int n = 0; n < 3; ++n) {
        o->rows_per_order[n] = op->row_begin[n + 1] - op->row_begin[n];
        o->delay_min[n] = op->dmin[n];
        o->delay_max[n] = op->dmax[n];
    }
    o->n_nodes = op->n_nodes;
    o->n_hats = op->time.n_hats;
    o->n_frames = op->time.n_frames;
    o->s_ref = op->s_ref;
    o->scale = op->scale;
    o->total_rows = op->total_rows;
    o->weight_precision = op->weight_precision;
    for (int n = 0; n < 3; ++n)
        o->total_rows_per_order[n] = op->total_row_begin[n + 1] - op->total_row_begin[n];
    o->shard_row_begin = op->shard_row_begin;
    o->shard_index = op->shard_index;
    o->shard_count = op->shard_count;
    return RTT_OK;
}

rtt_status rtt_op_status(rtt_op op, int32_t* flags_out, int clear, void* stream) {
    if (!op || !flags_out) {
        set_error("null argument");
        return RTT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int v = 0;
    RTT_CUDA(cudaMemcpyAsync(&v, op->dev_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RTT_CUDA(cudaStreamSynchronize(st));
    if (clear) RTT_CUDA(cudaMemsetAsync(op->dev_status, 0, sizeof(int), st));
    *flags_out = v;
    return RTT_OK;
}

rtt_status rtt_arm_rows(rtt_op op, int mask, int64_t* rows) {
    if (!op || !rows) {
        set_error("null argument");
        return RTT_EINVAL;
    }
    ArmSeg s;
    RTT_TRY(make_seg(op, mask, &s));
    *rows = s.total;
    return RTT_OK;
}

rtt_status rtt_apply_A(rtt_op op, const float* x, float* y, int batch, int mask, void* stream) {
    return apply_common<float>(op, x, y, batch, mask, stream, false);
}
rtt_status rtt_apply_A_AT(rtt_op op, const float* x, const float* d, float* y, float* g, int batch,
                          int mask, void* stream) {
    if (!op || batch < 1 || !x || !g) {
        set_error("invalid argument (op=%p batch=%d x=%p g=%p)", (void*)op, batch, (const void*)x,
                  (void*)g);
        return RTT_EINVAL;
    }
    ArmSeg seg;
    RTT_TRY(make_seg(op, mask, &seg));
    if (seg.total > 0 && !y) {
        set_error("null y with %d arm rows", seg.total);
        return RTT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    RTT_TRY(ensure_adjoint_scratch(op, batch, (int)sizeof(float)));
    cudaError_t e = launch_forward<float>(op, x, y, batch, seg, st);
    const float* r = y;
    const int64_t n = (int64_t)seg.total * op->time.n_frames * batch;
    if (e == cudaSuccess && d && n > 0) {
        const size_t bytes = (size_t)n * sizeof(float);
        if (bytes > op->rscratch_bytes) {
            if (op->rscratch) {
                cudaStreamSynchronize(st);
                cudaFree(op->rscratch);
                op->rscratch = nullptr;
                op->rscratch_bytes = 0;
            }
            if (cudaMalloc(&op->rscratch, bytes) != cudaSuccess) {
                op->rscratch = nullptr;
                set_error("residual scratch of %zu bytes: allocation failed", bytes);
                return RTT_ENOMEM;
            }
            op->rscratch_bytes = bytes;
        }
        residual_kernel<<<blocks(n < ((int64_t)1 << 24) ? n : ((int64_t)1 << 24)), 256, 0, st>>>(
            y, d, (float*)op->rscratch, n);
        e = cudaGetLastError();
        r = (const float*)op->rscratch;
    }
    if (e == cudaSuccess) e = launch_adjoint<float>(op, r, g, batch, seg, st);
    if (e != cudaSuccess) {
        set_error("apply launch failed: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    return RTT_OK;
}

rtt_status rtt_apply_AT(rtt_op op, const float* y, float* x, int batch, int mask, void* stream) {
    return apply_common<float>(op, y, x, batch, mask, stream, true);
}
rtt_status rtt_apply_A_f64(rtt_op op, const double* x, double* y, int batch, int mask,
                           void* stream) {
    return apply_common<double>(op, x, y, batch, mask, stream, false);
}
rtt_status rtt_apply_AT_f64(rtt_op op, const double* y, double* x, int batch, int mask,
                            void* stream) {
    return apply_common<double>(op, y, x, batch, mask, stream, true);
}

void rtt_destroy(rtt_op op) { free_op(op); }

}  // extern "C"
