// Age-localised probe information, anchor-connected reach and old-age
// innovation (Sec. 3.3 Eq. 10-13; Sec. 4.4 Eq. 29-30; Sec. 4.5 Eq. 35).
//
// I(a) = scale^2 sum_{rows of the arm, f} ( sum_{e in row} w_e / N_h
//        exp(-(t_o(f) - Delta_e + a)^2 / (2 h^2)) )^2, the probe evaluated
// directly at each ray's source point (not through the grid or the hats).
// One thread per (row, frame); per age the warp sums its squares with
// shuffles and lane 0 accumulates in FP64; blocks write FP64 partials that
// a second kernel adds in a fixed order (deterministic).  The fast pass
// evaluates the exponentials in FP32; ages whose value falls within 1e-3
// (relative) of the threshold rho^2 are evaluated again in FP64 so that the
// pass/fail decision is taken at FP64 accuracy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cub/cub.cuh>
#include <mutex>
#include <vector>

#include "rtt_internal.cuh"

namespace rtt {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocks = 1184;  // fixed grid (8 x 148): deterministic partials
constexpr int kMaxAges = 256;

struct ProbeArgs {
    const int32_t* row_ptr;
    const double* delay;
    const double* weight;
    ArmSeg seg;
    int Tn;
    double t0, cadence;
    double inv_2h2;
    double inv_Nh;
    int n_ages;
    const double* ages;  // device
    double* partial;     // [blocks][n_ages]
};

// one (operator, arm) job of the batched probe passes
struct ProbeJob {
    ProbeArgs p;      // p.partial: the partials of all jobs, block-major
    double scale2;    // scale^2 of the operator
    double thr;       // rho^2
    int blk0, nblk;   // the job's blocks in the flattened grid
};
constexpr int kProbeItemsPerBlock = 4096;  // (row, frame) items per block of the batched pass

template <typename T>
__device__ __forceinline__ T expo(T x);
template <>
__device__ __forceinline__ float expo<float>(float x) { return __expf(x); }
template <>
__device__ __forceinline__ double expo<double>(double x) { return exp(x); }

// The squared responses of the 32 (row, frame) items base + lane (those
// below n_items) for every age, or only the ages flagged in `mask`, summed
// over the warp; lane 0 adds each sum to acc[age].
template <typename T>
__device__ __forceinline__ void probe_warp(const ProbeArgs& p, int64_t base, int64_t n_items, int lane,
                                           double* acc, const uint8_t* mask) {
    const int64_t item = base + lane;
    const bool live = item < n_items;
    int row = 0, f = 0;
    if (live) {
        const int row_out = (int)(item / p.Tn);
        f = (int)(item - (int64_t)row_out * p.Tn);
        int r = row_out;
        for (int i = 0; i < p.seg.n; ++i) {
            if (r < p.seg.len[i]) {
                row = p.seg.begin[i] + r;
                break;
            }
            r -= p.seg.len[i];
        }
    }
    const double t = p.t0 + p.cadence * (double)f;
    const int e0 = live ? p.row_ptr[row] : 0, e1 = live ? p.row_ptr[row + 1] : 0;
    if constexpr (sizeof(T) == 4) {
        // FP32 path: t - Delta_e split once per (frame, ray) into a head
        // and a tail in FP32, so that x = (head + a) + tail needs only FP32
        // adds per age (head + a is exact near the cancellation x ~ 0,
        // and the ages are exact in FP32)
        constexpr int kRaysReg = 8;
        float hd[kRaysReg], tl[kRaysReg], wf[kRaysReg];
        const int nr = e1 - e0 < kRaysReg ? e1 - e0 : kRaysReg;
#pragma unroll
        for (int q = 0; q < kRaysReg; ++q) {
            hd[q] = 0.0f;
            tl[q] = 0.0f;
            wf[q] = 0.0f;
            if (q < nr) {
                const double b = t - p.delay[e0 + q];
                hd[q] = (float)b;
                tl[q] = (float)(b - (double)hd[q]);
                wf[q] = (float)(p.weight[e0 + q] * p.inv_Nh);
            }
        }
        const float i2h2 = (float)p.inv_2h2;
        for (int ia = 0; ia < p.n_ages; ++ia) {
            if (mask && !mask[ia]) continue;
            const float af = (float)p.ages[ia];
            float v = 0.0f;
#pragma unroll
            for (int q = 0; q < kRaysReg; ++q) {
                if (q < nr) {
                    const float x = (hd[q] + af) + tl[q];
                    const float arg = x * x * i2h2;
                    if (arg < 100.0f) v += wf[q] * __expf(-arg);
                }
            }
            for (int e = e0 + kRaysReg; e < e1; ++e) {  // rows with more rays
                const float x = (float)((t - p.delay[e]) + p.ages[ia]);
                const float arg = x * x * i2h2;
                if (arg < 100.0f) v += (float)(p.weight[e] * p.inv_Nh) * __expf(-arg);
            }
            float sq = v * v;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0) acc[ia] += (double)sq;
        }
    } else {
        for (int ia = 0; ia < p.n_ages; ++ia) {
            if (mask && !mask[ia]) continue;
            const double a = p.ages[ia];
            T v = T(0);
            for (int e = e0; e < e1; ++e) {
                const T x = (T)((t - p.delay[e]) + a);
                const T arg = x * x * (T)p.inv_2h2;
                if (arg < T(100)) v += (T)(p.weight[e] * p.inv_Nh) * expo<T>(-arg);
            }
            T sq = v * v;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0) acc[ia] += (double)sq;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) probe_kernel(const ProbeArgs p) {
    __shared__ double acc[kProbeThreads / 32][kMaxAges];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int a = lane; a < p.n_ages; a += 32) acc[warp][a] = 0.0;
    __syncwarp();
    const int64_t n_items = (int64_t)p.seg.total * p.Tn;
    // warp-contiguous (row, frame) items; every warp of the grid walks the
    // same fixed sequence so the partial sums do not depend on timing
    const int64_t warps_total = (int64_t)gridDim.x * (kProbeThreads / 32);
    const int64_t gw = (int64_t)blockIdx.x * (kProbeThreads / 32) + warp;
    for (int64_t base = gw * 32; base < n_items; base += warps_total * 32)
        probe_warp<T>(p, base, n_items, lane, acc[warp], nullptr);
    __syncthreads();
    for (int a = threadIdx.x; a < p.n_ages; a += kProbeThreads) {
        double s = 0.0;
        for (int w = 0; w < kProbeThreads / 32; ++w) s += acc[w][a];
        p.partial[(int64_t)blockIdx.x * p.n_ages + a] = s;
    }
}

// ---- the probes of many (operator, arm) jobs in one launch per pass: the
// jobs' (row, frame) items cut into blocks of kProbeItemsPerBlock, all blocks
// in one grid (a block finds its job by binary search on the first blocks)
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) probe_multi_kernel(const ProbeJob* __restrict__ jobs,
                                                                    int n_jobs,
                                                                    const uint8_t* __restrict__ flags) {
    __shared__ double acc[kProbeThreads / 32][kMaxAges];
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].blk0 <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ProbeArgs p = jobs[lo].p;
    const int lb = (int)blockIdx.x - jobs[lo].blk0;
    const uint8_t* mask = flags ? flags + (int64_t)lo * p.n_ages : nullptr;
    if (mask) {  // the FP64 pass: only jobs with an age near the threshold
        bool any = false;
        for (int a = 0; a < p.n_ages; ++a) any = any || mask[a];
        if (!any) return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int a = lane; a < p.n_ages; a += 32) acc[warp][a] = 0.0;
    __syncwarp();
    const int64_t n_items = (int64_t)p.seg.total * p.Tn;
    const int64_t i0 = (int64_t)lb * kProbeItemsPerBlock;
    const int64_t i1 = i0 + kProbeItemsPerBlock < n_items ? i0 + kProbeItemsPerBlock : n_items;
    for (int64_t base = i0 + warp * 32; base < i1; base += kProbeThreads)
        probe_warp<T>(p, base, i1, lane, acc[warp], mask);
    __syncthreads();
    for (int a = threadIdx.x; a < p.n_ages; a += kProbeThreads) {
        double s = 0.0;
        for (int w = 0; w < kProbeThreads / 32; ++w) s += acc[w][a];
        p.partial[(int64_t)blockIdx.x * p.n_ages + a] = s;
    }
}

// info[j][a] = scale^2 x the job's block partials summed in order.  Pass 0
// (FP32 values) also sets flags[j][a] where the value is within 1e-3 of
// rho^2; pass 1 (FP64 values) replaces just the flagged entries.
__global__ void probe_multi_reduce(const ProbeJob* __restrict__ jobs, int n_jobs, int n_ages,
                                   const double* __restrict__ partial, double* info, uint8_t* flags,
                                   int pass) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_jobs * n_ages) return;
    const int j = t / n_ages, a = t - j * n_ages;
    if (pass == 1 && !flags[t]) return;
    double s = 0.0;
    for (int b = 0; b < jobs[j].nblk; ++b) s += partial[(int64_t)(jobs[j].blk0 + b) * n_ages + a];
    const double v = jobs[j].scale2 * s;
    info[t] = v;
    if (pass == 0) flags[t] = fabs(v - jobs[j].thr) <= 1e-3 * jobs[j].thr ? 1 : 0;
}

__global__ void probe_reduce(const double* partial, int n_blocks, int n_ages, double scale2,
                             double* out) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_ages) return;
    double s = 0.0;
    for (int b = 0; b < n_blocks; ++b) s += partial[(int64_t)b * n_ages + a];
    out[a] = scale2 * s;
}

// Direct (ray, frame) ages Delta_e - t_o(f) with throughput weights.
__global__ void direct_ages(int64_t n_rays0, int Tn, double t0, double cadence,
                            const double* delay, const double* thr, double* key, double* val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rays0 * Tn) return;
    const int64_t e = i / Tn;
    const int f = (int)(i - e * Tn);
    key[i] = delay[e] - (t0 + cadence * (double)f);
    val[i] = thr[e];
}

__global__ void first_reaching(int64_t n, const double* cum, double target, int64_t* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cum[i] >= target && (i == 0 || cum[i - 1] < target)) *out = i;
}


// the probe arguments of one operator and arm (Eq. 10-12: N_h from the
// source annulus area and the probe width h)
static ProbeArgs probe_args(const rtt_op_s* op, const ArmSeg& seg, int n_ages, const double* ages_dev,
                            double h, double* partial) {
    ProbeArgs p{};
    p.row_ptr = op->row_ptr;
    p.delay = op->delay;
    p.weight = op->weight;
    p.seg = seg;
    p.Tn = op->time.n_frames;
    p.t0 = op->time.t0;
    p.cadence = op->time.cadence;
    p.inv_2h2 = 1.0 / (2.0 * h * h);
    const double Nh = std::sqrt(M_PI * (op->grid.r_out * op->grid.r_out -
                                        op->grid.r_in * op->grid.r_in) * h * std::sqrt(M_PI));
    p.inv_Nh = 1.0 / Nh;
    p.n_ages = n_ages;
    p.ages = ages_dev;
    p.partial = partial;
    return p;
}

// ---- batched probes of many (operator, arm) jobs: all buffers allocated
// once here; a run is four launches on one stream, no host synchronisation
struct ProbePlan {
    int n_jobs = 0, n_ages = 0, blocks = 0;
    double* ages = nullptr;
    double* partial = nullptr;
    double* info = nullptr;
    uint8_t* flags = nullptr;
    ProbeJob* jobs = nullptr;
};

void probe_plan_destroy(ProbePlan* pp) {
    if (!pp) return;
    cudaFree(pp->ages);
    cudaFree(pp->partial);
    cudaFree(pp->info);
    cudaFree(pp->flags);
    cudaFree(pp->jobs);
    delete pp;
}

rtt_status probe_plan_create(const rtt_op_s* const* job_ops, const ArmSeg* segs, int n_jobs, int n_ages,
                             const double* ages_host, double h, ProbePlan** out) {
    *out = nullptr;
    if (n_jobs < 1 || n_ages < 1 || n_ages > kMaxAges) {
        set_error("probe plan: %d jobs, %d ages (1..%d)", n_jobs, n_ages, kMaxAges);
        return RTT_EINVAL;
    }
    ProbePlan* pp = new (std::nothrow) ProbePlan();
    if (!pp) {
        set_error("probe plan: host allocation failed");
        return RTT_ENOMEM;
    }
    pp->n_jobs = n_jobs;
    pp->n_ages = n_ages;
    std::vector<ProbeJob> jobs(n_jobs);
    int blocks = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const rtt_op_s* op = job_ops[j];
        const int64_t items = (int64_t)segs[j].total * op->time.n_frames;
        jobs[j].nblk = (int)((items + kProbeItemsPerBlock - 1) / kProbeItemsPerBlock);
        if (jobs[j].nblk < 1) jobs[j].nblk = 1;
        jobs[j].blk0 = blocks;
        blocks += jobs[j].nblk;
        jobs[j].scale2 = op->scale * op->scale;
        jobs[j].thr = op->opt.rho * op->opt.rho;
    }
    pp->blocks = blocks;
    cudaError_t e = cudaMalloc(&pp->ages, (size_t)n_ages * 8);
    if (e == cudaSuccess) e = cudaMalloc(&pp->partial, (size_t)blocks * n_ages * 8);
    if (e == cudaSuccess) e = cudaMalloc(&pp->info, (size_t)n_jobs * n_ages * 8);
    if (e == cudaSuccess) e = cudaMalloc(&pp->flags, (size_t)n_jobs * n_ages);
    if (e == cudaSuccess) e = cudaMalloc(&pp->jobs, sizeof(ProbeJob) * n_jobs);
    if (e != cudaSuccess) {
        probe_plan_destroy(pp);
        set_error("probe plan: device allocation failed");
        return RTT_ENOMEM;
    }
    for (int j = 0; j < n_jobs; ++j) jobs[j].p = probe_args(job_ops[j], segs[j], n_ages, pp->ages, h, pp->partial);
    e = cudaMemcpy(pp->ages, ages_host, (size_t)n_ages * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pp->jobs, jobs.data(), sizeof(ProbeJob) * n_jobs, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        probe_plan_destroy(pp);
        set_error("probe plan: copy failed");
        return RTT_ECUDA;
    }
    *out = pp;
    return RTT_OK;
}

cudaError_t probe_plan_run(ProbePlan* pp, cudaStream_t st) {
    const int n = pp->n_jobs * pp->n_ages;
    probe_multi_kernel<float><<<pp->blocks, kProbeThreads, 0, st>>>(pp->jobs, pp->n_jobs, nullptr);
    probe_multi_reduce<<<(n + 127) / 128, 128, 0, st>>>(pp->jobs, pp->n_jobs, pp->n_ages, pp->partial,
                                                        pp->info, pp->flags, 0);
    probe_multi_kernel<double><<<pp->blocks, kProbeThreads, 0, st>>>(pp->jobs, pp->n_jobs, pp->flags);
    probe_multi_reduce<<<(n + 127) / 128, 128, 0, st>>>(pp->jobs, pp->n_jobs, pp->n_ages, pp->partial,
                                                        pp->info, pp->flags, 1);
    return cudaGetLastError();
}

const double* probe_plan_info(const ProbePlan* pp) { return pp->info; }

static rtt_status run_probe(const rtt_op_s* op, const ArmSeg& seg, int n_ages,
                            const double* ages_h, double h, bool fp64, double* info_h,
                            cudaStream_t st) {
    if (n_ages == 0) return RTT_OK;
    double *d_ages = nullptr, *d_part = nullptr, *d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_ages, n_ages * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_part, (size_t)kProbeBlocks * n_ages * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, n_ages * 8);
    if (e != cudaSuccess) {
        cudaFree(d_ages);
        cudaFree(d_part);
        cudaFree(d_out);
        set_error("probe scratch allocation failed: %s", cudaGetErrorString(e));
        return RTT_ENOMEM;
    }
    const ProbeArgs p = probe_args(op, seg, n_ages, d_ages, h, d_part);
    e = cudaMemcpyAsync(d_ages, ages_h, n_ages * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        if (fp64)
            probe_kernel<double><<<kProbeBlocks, kProbeThreads, 0, st>>>(p);
        else
            probe_kernel<float><<<kProbeBlocks, kProbeThreads, 0, st>>>(p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        probe_reduce<<<(n_ages + 127) / 128, 128, 0, st>>>(d_part, kProbeBlocks, n_ages,
                                                           op->scale * op->scale, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(info_h, d_out, n_ages * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_ages);
    cudaFree(d_part);
    cudaFree(d_out);
    if (e != cudaSuccess) {
        set_error("probe kernels failed: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    return RTT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  The per-block partial sums live in a file-scope
// device array that every GPU loading the library holds until the process
// exits; the host side only needs its device address, looked up once per
// device.  Each launch overwrites every partial it later reads, so nothing
// has to be cleared between calls, but two calls in flight at the same time
// (on different streams) share the array and race.
// ---------------------------------------------------------------------------
constexpr int kStaticProbeAges = kMaxAges;
static __device__ __align__(256) double g_probe_partial[kProbeBlocks * kStaticProbeAges];

constexpr int kMaxDevices = 64;
static double* g_probe_partial_addr[kMaxDevices];
static std::mutex g_probe_partial_mu;

static rtt_status static_partial_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("cudaGetDevice: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device %d beyond the %d devices the static scratch table covers", dev,
                  kMaxDevices);
        return RTT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_probe_partial_mu);
    if (!g_probe_partial_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_probe_partial);
        if (e != cudaSuccess || !ptr) {
            set_error("cudaGetSymbolAddress(static probe scratch): %s", cudaGetErrorString(e));
            return RTT_ECUDA;
        }
        g_probe_partial_addr[dev] = static_cast<double*>(ptr);
    }
    *out = g_probe_partial_addr[dev];
    return RTT_OK;
}

}  // namespace rtt

using namespace rtt;

extern "C" rtt_status rtt_probe_info_noalloc(rtt_op op, int arm_mask, int n_ages,
                                             const double* ages_dev, double h, double* info_dev,
                                             void* stream) {
    if (!op || !(h > 0.0) || n_ages < 0 || (n_ages > 0 && (!ages_dev || !info_dev))) {
        set_error("invalid probe arguments (n_ages=%d, h=%g)", n_ages, h);
        return RTT_EINVAL;
    }
    if (n_ages > kStaticProbeAges) {
        set_error("rtt_probe_info_noalloc: %d ages exceed the static scratch limit of %d", n_ages,
                  kStaticProbeAges);
        return RTT_EINVAL;
    }
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s != RTT_OK) return s;
    if (n_ages == 0) return RTT_OK;
    double* partial = nullptr;
    s = static_partial_address(&partial);
    if (s != RTT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const ProbeArgs p = probe_args(op, seg, n_ages, ages_dev, h, partial);
    probe_kernel<float><<<kProbeBlocks, kProbeThreads, 0, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        probe_reduce<<<(n_ages + 127) / 128, 128, 0, st>>>(partial, kProbeBlocks, n_ages,
                                                           op->scale * op->scale, info_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("probe kernels failed: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    return RTT_OK;
}

extern "C" rtt_status rtt_probe_info(rtt_op op, int arm_mask, int n_ages, const double* ages,
                                     double h, double* info, void* stream) {
    if (!op || n_ages < 0 || n_ages > kMaxAges || (n_ages > 0 && (!ages || !info)) || !(h > 0.0)) {
        set_error("invalid probe arguments (n_ages=%d, h=%g)", n_ages, h);
        return RTT_EINVAL;
    }
    ArmSeg seg;
    rtt_status s = make_seg(op, arm_mask, &seg);
    if (s != RTT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    s = run_probe(op, seg, n_ages, ages, h, false, info, st);
    if (s != RTT_OK) return s;
    // FP64 re-evaluation of the ages near the detection threshold
    const double thr = op->opt.rho * op->opt.rho;
    std::vector<double> amb_age;
    std::vector<int> amb_idx;
    for (int i = 0; i < n_ages; ++i) {
        if (std::fabs(info[i] - thr) <= 1e-3 * thr) {
            amb_age.push_back(ages[i]);
            amb_idx.push_back(i);
        }
    }
    if (!amb_age.empty()) {
        std::vector<double> v(amb_age.size());
        s = run_probe(op, seg, (int)amb_age.size(), amb_age.data(), h, true, v.data(), st);
        if (s != RTT_OK) return s;
        for (size_t j = 0; j < v.size(); ++j) info[amb_idx[j]] = v[j];
    }
    return RTT_OK;
}

extern "C" rtt_status rtt_direct_age_quantile(rtt_op op, double q, double* out, void* stream) {
    if (!op || !out || !(q > 0.0 && q <= 1.0)) {
        set_error("invalid quantile arguments");
        return RTT_EINVAL;
    }
    RTT_TRY(whole_only(op, "the direct age quantile"));
    cudaStream_t st = (cudaStream_t)stream;
    // direct rays are the rays of rows [0, row_begin[1]): rays [0, row_ptr[row_begin[1]])
    int32_t n0 = 0;
    cudaError_t e = cudaMemcpyAsync(&n0, op->row_ptr + op->row_begin[1], 4,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("quantile: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    const int64_t n = (int64_t)n0 * op->time.n_frames;
    double *k_in = nullptr, *k_out = nullptr, *v_in = nullptr, *v_out = nullptr, *cum = nullptr;
    int64_t* d_idx = nullptr;
    void* tmp = nullptr;
    size_t tb1 = 0, tb2 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb1, k_in, k_out, v_in, v_out, n, 0, 64, st);
    cub::DeviceScan::InclusiveSum(nullptr, tb2, v_out, cum, n, st);
    const size_t tb = tb1 > tb2 ? tb1 : tb2;
    e = cudaMalloc(&k_in, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&k_out, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&v_in, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&v_out, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&cum, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_idx, 8);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, tb + 16);
    double total = 0.0, age = 0.0;
    int64_t idx = -1;
    if (e == cudaSuccess) {
        direct_ages<<<(int)((n + 255) / 256), 256, 0, st>>>(n0, op->time.n_frames, op->time.t0,
                                                              op->time.cadence, op->delay, op->thr,
                                                              k_in, v_in);
        e = cudaGetLastError();
    }
    size_t t1 = tb;
    if (e == cudaSuccess) e = cub::DeviceRadixSort::SortPairs(tmp, t1, k_in, k_out, v_in, v_out, n, 0, 64, st);
    t1 = tb;
    if (e == cudaSuccess) e = cub::DeviceScan::InclusiveSum(tmp, t1, v_out, cum, n, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, cum + (n - 1), 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_idx, 0xff, 8, st);
    if (e == cudaSuccess) {
        first_reaching<<<(int)((n + 255) / 256), 256, 0, st>>>(n, cum, q * total, d_idx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&idx, d_idx, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        if (idx < 0) idx = n - 1;
        e = cudaMemcpyAsync(&age, k_out + idx, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFree(k_in);
    cudaFree(k_out);
    cudaFree(v_in);
    cudaFree(v_out);
    cudaFree(cum);
    cudaFree(d_idx);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        set_error("quantile kernels failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RTT_ENOMEM : RTT_ECUDA;
    }
    *out = age;
    return RTT_OK;
}

// Anchor-connected reach and old-age innovation from I(a) (host logic on
// the per-order delay ranges the operator recorded).
extern "C" rtt_status rtt_reach(rtt_op op, int arm_mask, int n_ages, const double* ages,
                                const double* info, double h, double a0q, double age_step,
                                rtt_reach_result* out, uint8_t* pass) {
    if (!op || !out || n_ages < 1 || !ages || !info || !(h > 0.0) || !(age_step > 0.0) ||
        arm_mask < 1 || arm_mask > 7) {
        set_error("invalid reach arguments");
        return RTT_EINVAL;
    }
    RTT_TRY(whole_only(op, "reach"));
    const double thr = op->opt.rho * op->opt.rho;
    const double to_min = op->time.t0;
    const double to_max = op->time.t0 + op->time.cadence * (op->time.n_frames - 1);
    // footprint intervals W_n = [t_o,min - Delta_n^max, t_o,max - Delta_n^min]
    std::vector<std::pair<double, double>> W;
    for (int n = 0; n < 3; ++n) {
        if (!(arm_mask & (1 << n))) continue;
        if (op->row_begin[n + 1] == op->row_begin[n]) continue;
        W.push_back({to_min - op->dmax[n], to_max - op->dmin[n]});
    }
    std::sort(W.begin(), W.end());
    auto covered = [&](double lo, double hi) {
        double cur = lo;
        for (auto& iv : W) {
            if (iv.first > cur) break;
            cur = std::max(cur, iv.second);
            if (cur >= hi) return true;
        }
        return cur >= hi;
    };
    int anchor = -1;
    for (int i = 0; i < n_ages; ++i) {
        if (covered(-ages[i] - 3.0 * h, -ages[i] + 3.0 * h)) {
            anchor = i;
            break;
        }
    }
    double L = 0.0;
    if (anchor >= 0 && info[anchor] >= thr) {
        int j = anchor;
        while (j + 1 < n_ages && info[j + 1] >= thr) ++j;
        L = ages[j] - ages[anchor];
    }
    double treach = NAN;
    for (int i = 0; i < n_ages; ++i)
        if (info[i] >= thr) treach = ages[i];
    double J = 0.0;
    for (int i = 0; i < n_ages; ++i)
        if (ages[i] > a0q) J += std::log1p(info[i]);
    out->anchor_index = anchor;
    out->anchor_age = anchor >= 0 ? ages[anchor] : NAN;
    out->L_anchor = L;
    out->T_reach = treach;
    out->A0q = a0q;
    out->J_old = age_step * J;
    if (pass)
        for (int i = 0; i < n_ages; ++i) pass[i] = info[i] >= thr ? 1 : 0;
    return RTT_OK;
}
