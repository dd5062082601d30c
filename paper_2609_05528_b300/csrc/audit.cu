// Multi-geometry audit (Sec. 6.2-6.3): for each operator (geometry)
// and each observation arm, the age probes, anchor-connected reach, direct
// age boundary and old-age innovation, and the restricted Gram spectrum with
// its operational rank.  Host orchestration of the library's kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "rtt_internal.cuh"

using namespace rtt;

extern "C" rtt_status rtt_gram(rtt_op op, int arm_mask, const double* Q, int d, double* G,
                               void* stream);
extern "C" rtt_status rtt_gram_normal(rtt_op op, int arm_mask, const double* Q, int d, double* G,
                                      void* stream);
extern "C" rtt_status rtt_eig_sym(int n, double* A, double* evals_host, double* V, int max_sweeps,
                                  int* sweeps_host, void* stream);
extern "C" rtt_status rtt_probe_info(rtt_op op, int arm_mask, int n_ages, const double* ages,
                                     double h, double* info, void* stream);
extern "C" rtt_status rtt_direct_age_quantile(rtt_op op, double q, double* out, void* stream);
extern "C" rtt_status rtt_reach(rtt_op op, int arm_mask, int n_ages, const double* ages,
                                const double* info, double h, double a0q, double age_step,
                                rtt_reach_result* out, uint8_t* pass);

extern "C" rtt_status rtt_gram_class(rtt_op op, int arm_mask, int kind, double* G, void* stream);

extern "C" rtt_status rtt_eigvals_sym_batched(int n, int batch, double* A, double* evals_host,
                                              void* stream);

extern "C" rtt_status rtt_eig_sym_batched(int n, int batch, double* A, double* evals_host,
                                          double* V, int max_sweeps, int* sweeps_host,
                                          void* stream);

extern "C" rtt_status rtt_operational_rank(int n, const double* evals, double rho, int* rank_out,
                                           double* margin_out, double* sigma_out) {
    if (n < 1 || !evals || !rank_out || !margin_out || !(rho > 0.0) || !std::isfinite(rho)) {
        set_error("invalid operational-rank arguments (n=%d, rho=%g)", n, rho);
        return RTT_EINVAL;
    }
    std::vector<double> sig(n);
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(evals[i])) {
            set_error("operational rank: eigenvalue %d is not finite", i);
            return RTT_EINVAL;
        }
        sig[i] = std::sqrt(evals[i] > 0.0 ? evals[i] : 0.0);
    }
    std::sort(sig.begin(), sig.end(), [](double a, double c) { return a > c; });
    int rank = 0;
    double margin = INFINITY;
    for (int i = 0; i < n; ++i) {
        if (sig[i] >= rho) ++rank;
        margin = std::fmin(margin, std::fabs(sig[i] - rho) / rho);
    }
    *rank_out = rank;
    *margin_out = margin;
    if (sigma_out) std::copy(sig.begin(), sig.end(), sigma_out);
    return RTT_OK;
}

// ---------------------------------------------------------------------------
// Batched audit plan: every (geometry, arm) job of the class-Gram audit in one
// launch per stage (probes: FP32 pass, FP64 re-check of ages near rho^2;
// class Gram tiles and their reduction; eigenvalues), everything allocated
// and every per-geometry table built at creation, so that a run enqueues
// device work only (it can be captured in a CUDA graph) and the results call
// synchronises once.
// ---------------------------------------------------------------------------
struct rtt_audit_plan_s {
    std::vector<rtt_op> ops;
    std::vector<int> arms;
    std::vector<double> ages;
    double h = 0.0;
    int n_jobs = 0, d = 224;
    std::vector<double> a0q;  // A_{0,q} per geometry
    ProbePlan* probes = nullptr;
    ClassPlan* grams = nullptr;
    double *G = nullptr, *V = nullptr, *ed = nullptr, *ee = nullptr, *ework = nullptr, *ev = nullptr;
    cudaEvent_t t[4] = {nullptr, nullptr, nullptr, nullptr};
    bool ran = false;
};

static void plan_free(rtt_audit_plan_s* p) {
    if (!p) return;
    probe_plan_destroy(p->probes);
    class_plan_destroy(p->grams);
    void* ps[] = {p->G, p->V, p->ed, p->ee, p->ework, p->ev};
    for (void* q : ps) cudaFree(q);
    for (cudaEvent_t e : p->t)
        if (e) cudaEventDestroy(e);
    delete p;
}

extern "C" rtt_status rtt_audit_plan_create(const rtt_op* ops, int n_ops, const int* arm_masks, int n_arms,
                                            int n_ages, const double* ages_host, double h, double quantile,
                                            int class_kind, void* stream, rtt_audit_plan* out) {
    if (!out || !ops || n_ops < 1 || !arm_masks || n_arms < 1 || n_ages < 1 || n_ages > 256 || !ages_host ||
        !(h > 0.0) || !(quantile > 0.0 && quantile <= 1.0) ||
        (class_kind != RTT_CLASS_S224 && class_kind != RTT_CLASS_L224)) {
        set_error("invalid audit-plan arguments");
        return RTT_EINVAL;
    }
    *out = nullptr;
    for (int g = 0; g < n_ops; ++g) {
        if (!ops[g]) {
            set_error("audit plan: operator %d missing", g);
            return RTT_EINVAL;
        }
        RTT_TRY(whole_only(ops[g], "the rank audit"));
    }
    cudaStream_t st = (cudaStream_t)stream;
    rtt_audit_plan_s* p = new (std::nothrow) rtt_audit_plan_s();
    if (!p) {
        set_error("audit plan: host allocation failed");
        return RTT_ENOMEM;
    }
    p->ops.assign(ops, ops + n_ops);
    p->arms.assign(arm_masks, arm_masks + n_arms);
    p->ages.assign(ages_host, ages_host + n_ages);
    p->h = h;
    p->n_jobs = n_ops * n_arms;
    const int nb = p->n_jobs, d = p->d;
    std::vector<ArmSeg> segs(nb);
    std::vector<const rtt_op_s*> job_ops(nb);
    std::vector<int> job_op(nb);
    rtt_status s = RTT_OK;
    for (int g = 0; g < n_ops && s == RTT_OK; ++g)
        for (int a = 0; a < n_arms && s == RTT_OK; ++a) {
            const int j = g * n_arms + a;
            s = make_seg(ops[g], arm_masks[a], &segs[j]);
            job_ops[j] = ops[g];
            job_op[j] = g;
        }
    p->a0q.resize(n_ops);
    for (int g = 0; g < n_ops && s == RTT_OK; ++g) s = rtt_direct_age_quantile(ops[g], quantile, &p->a0q[g], stream);
    if (s == RTT_OK) s = probe_plan_create(job_ops.data(), segs.data(), nb, n_ages, ages_host, h, &p->probes);
    const size_t gbytes = (size_t)nb * d * d * 8;
    if (s == RTT_OK && (cudaMalloc(&p->G, gbytes) != cudaSuccess || cudaMalloc(&p->V, gbytes) != cudaSuccess ||
                        cudaMalloc(&p->ed, (size_t)nb * d * 8) != cudaSuccess ||
                        cudaMalloc(&p->ee, (size_t)nb * d * 8) != cudaSuccess ||
                        cudaMalloc(&p->ework, (size_t)nb * 2 * d * 8) != cudaSuccess ||
                        cudaMalloc(&p->ev, (size_t)nb * d * 8) != cudaSuccess)) {
        set_error("audit plan: device allocation failed");
        s = RTT_ENOMEM;
    }
    if (s == RTT_OK)
        s = class_plan_create(p->ops.data(), n_ops, job_op.data(), segs.data(), nb, class_kind, p->G, st,
                              &p->grams);
    for (int i = 0; i < 4 && s == RTT_OK; ++i)
        if (cudaEventCreate(&p->t[i]) != cudaSuccess) {
            set_error("audit plan: event creation failed");
            s = RTT_ECUDA;
        }
    if (s != RTT_OK) {
        plan_free(p);
        return s;
    }
    *out = p;
    return RTT_OK;
}

extern "C" rtt_status rtt_audit_plan_run(rtt_audit_plan p, void* stream) {
    if (!p) {
        set_error("null audit plan");
        return RTT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = p->n_jobs, d = p->d;
    cudaError_t e = cudaEventRecord(p->t[0], st);
    if (e == cudaSuccess) e = probe_plan_run(p->probes, st);
    if (e == cudaSuccess) e = cudaEventRecord(p->t[1], st);
    if (e == cudaSuccess) e = class_plan_run(p->grams, st);
    if (e == cudaSuccess) e = cudaEventRecord(p->t[2], st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->V, p->G, (size_t)nb * d * d * 8, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = launch_eigvals_batched(d, nb, p->V, p->ed, p->ee, p->ework, p->ev, st);
    if (e == cudaSuccess) e = cudaEventRecord(p->t[3], st);
    if (e != cudaSuccess) {
        set_error("audit plan run: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    p->ran = true;
    return RTT_OK;
}

extern "C" rtt_status rtt_audit_plan_results(rtt_audit_plan p, rtt_audit_record* out, double* sigma_out,
                                             void* stream) {
    if (!p || !out) {
        set_error("invalid audit-plan results arguments");
        return RTT_EINVAL;
    }
    if (!p->ran) {
        set_error("audit plan: no run to read");
        return RTT_ESTATE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = p->n_jobs, d = p->d, n_ages = (int)p->ages.size(), n_arms = (int)p->arms.size();
    std::vector<double> info((size_t)nb * n_ages), ev((size_t)nb * d);
    cudaError_t e = cudaMemcpyAsync(info.data(), probe_plan_info(p->probes), info.size() * 8,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ev.data(), p->ev, ev.size() * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("audit plan results: %s", cudaGetErrorString(e));
        return RTT_ECUDA;
    }
    // stage times (0 where the events carry none, e.g. a run replayed from a
    // captured graph)
    float ms[3] = {0.f, 0.f, 0.f};
    for (int i = 0; i < 3; ++i)
        if (cudaEventElapsedTime(&ms[i], p->t[i], p->t[i + 1]) != cudaSuccess) {
            ms[i] = 0.f;
            (void)cudaGetLastError();
        }
    const double age_step = n_ages > 1 ? p->ages[1] - p->ages[0] : 1.0;
    std::vector<double> sig(d);
    for (int j = 0; j < nb; ++j) {
        rtt_op op = p->ops[j / n_arms];
        rtt_audit_record& r = out[j];
        r.arm_mask = p->arms[j % n_arms];
        rtt_status s = rtt_reach(op, r.arm_mask, n_ages, p->ages.data(), info.data() + (size_t)j * n_ages, p->h,
                                 p->a0q[j / n_arms], age_step, &r.reach, nullptr);
        if (s != RTT_OK) return s;
        // a spectrum with an eigenvalue within the reduction's error bound of
        // rho^2 is decided by the Jacobi spectrum of its Gram (relative accuracy)
        const double rho = op->opt.rho;
        double amax = 0.0;
        for (int i = 0; i < d; ++i) amax = std::fmax(amax, std::fabs(ev[(size_t)j * d + i]));
        const double bound = 64.0 * d * 2.220446049250313e-16 * amax;
        bool near = false;
        for (int i = 0; i < d; ++i) near = near || std::fabs(ev[(size_t)j * d + i] - rho * rho) <= bound;
        r.jacobi_sweeps = 0;
        if (near) {
            s = rtt_eig_sym(d, p->G + (size_t)j * d * d, ev.data() + (size_t)j * d, p->V, 80, &r.jacobi_sweeps,
                            stream);
            if (s != RTT_OK) return s;
        }
        int rank = 0;
        double margin = INFINITY, smin_pos = INFINITY;
        s = rtt_operational_rank(d, ev.data() + (size_t)j * d, rho, &rank, &margin, sig.data());
        if (s != RTT_OK) return s;
        for (int i = 0; i < d; ++i)
            if (sig[i] > 0.0) smin_pos = std::fmin(smin_pos, sig[i]);
        r.rank = rank;
        r.margin = margin;
        r.sigma_max = sig[0];
        r.sigma_min_pos = smin_pos;
        r.s_ref = op->s_ref;
        // stage times of the whole batch, shared evenly by its records
        r.seconds_probe = 1e-3 * ms[0] / nb;
        r.seconds_gram = 1e-3 * ms[1] / nb;
        r.seconds_eig = 1e-3 * ms[2] / nb;
        r.seconds = r.seconds_probe + r.seconds_gram + r.seconds_eig;
        if (sigma_out)
            for (int i = 0; i < d; ++i) sigma_out[(size_t)j * d + i] = sig[i];
    }
    return RTT_OK;
}

extern "C" rtt_status rtt_audit_plan_destroy(rtt_audit_plan p) {
    plan_free(p);
    return RTT_OK;
}

extern "C" rtt_status rtt_rank_audit(const rtt_op* ops, int n_ops, const double* const* Q_dev,
                                     int d, const int* arm_masks, int n_arms, int n_ages,
                                     const double* ages_host, double h, double quantile,
                                     int gram_mode, rtt_audit_record* out, double* sigma_out,
                                     void* stream) {
    if (!ops || n_ops < 1 || !Q_dev || d < 1 || d > 4096 || !arm_masks || n_arms < 1 ||
        gram_mode < RTT_GRAM_DATA || gram_mode > RTT_GRAM_CLASS_L224 ||
        (gram_mode >= RTT_GRAM_CLASS_S224 && d != 224) ||
        n_ages < 1 || n_ages > 256 || !ages_host || !(h > 0.0) || !(quantile > 0.0) || !out) {
        set_error("invalid rank-audit arguments");
        return RTT_EINVAL;
    }
    for (int g = 0; g < n_ops; ++g) RTT_TRY(whole_only(ops[g], "the rank audit"));
    if (gram_mode >= RTT_GRAM_CLASS_S224) {
        // the batched plan; a geometry with rows the class path does not
        // handle sends the whole audit down the per-geometry route below
        rtt_audit_plan plan = nullptr;
        rtt_status s = rtt_audit_plan_create(ops, n_ops, arm_masks, n_arms, n_ages, ages_host, h, quantile,
                                             gram_mode == RTT_GRAM_CLASS_S224 ? RTT_CLASS_S224 : RTT_CLASS_L224,
                                             stream, &plan);
        if (s == RTT_OK) {
            s = rtt_audit_plan_run(plan, stream);
            if (s == RTT_OK) s = rtt_audit_plan_results(plan, out, sigma_out, stream);
            rtt_audit_plan_destroy(plan);
            return s;
        }
        if (s != RTT_ESTATE) return s;
    }
    const int nb = n_ops * n_arms;
    double *G = nullptr, *V = nullptr;
    cudaError_t e = cudaMalloc(&G, (size_t)nb * d * d * 8);
    if (e == cudaSuccess) e = cudaMalloc(&V, (size_t)nb * d * d * 8);
    if (e != cudaSuccess) {
        cudaFree(G);
        cudaFree(V);
        set_error("rank audit: allocation failed");
        return RTT_ENOMEM;
    }
    std::vector<double> info(n_ages), ev((size_t)nb * d);
    std::vector<int> sweeps(nb);
    const double age_step = n_ages > 1 ? ages_host[1] - ages_host[0] : 1.0;
    rtt_status s = RTT_OK;
    // probes, reach and restricted Grams of every (geometry, arm)
    for (int g = 0; g < n_ops && s == RTT_OK; ++g) {
        rtt_op op = ops[g];
        if (!op || (!Q_dev[g] && gram_mode < RTT_GRAM_CLASS_S224)) {
            set_error("rank audit: operator or class %d missing", g);
            s = RTT_EINVAL;
            break;
        }
        double a0 = 0.0;
        s = rtt_direct_age_quantile(op, quantile, &a0, stream);
        for (int ai = 0; ai < n_arms && s == RTT_OK; ++ai) {
            const auto t0 = std::chrono::steady_clock::now();
            rtt_audit_record& r = out[(size_t)g * n_arms + ai];
            r.arm_mask = arm_masks[ai];
            s = rtt_probe_info(op, arm_masks[ai], n_ages, ages_host, h, info.data(), stream);
            if (s != RTT_OK) break;
            rtt_reach_result rr;
            s = rtt_reach(op, arm_masks[ai], n_ages, ages_host, info.data(), h, a0, age_step, &rr,
                          nullptr);
            if (s != RTT_OK) break;
            r.reach = rr;
            const auto t1 = std::chrono::steady_clock::now();
            double* Gi = G + ((size_t)g * n_arms + ai) * d * d;
            if (gram_mode >= RTT_GRAM_CLASS_S224) {
                s = rtt_gram_class(op, arm_masks[ai],
                                   gram_mode == RTT_GRAM_CLASS_S224 ? RTT_CLASS_S224 : RTT_CLASS_L224,
                                   Gi, stream);
                if (s == RTT_ESTATE) {  // rows the class path does not handle
                    s = Q_dev[g] ? rtt_gram_normal(op, arm_masks[ai], Q_dev[g], d, Gi, stream)
                                 : RTT_EINVAL;
                    if (s == RTT_EINVAL) set_error("rank audit: class Gram unavailable and no Q");
                }
            } else {
                s = gram_mode == RTT_GRAM_NORMAL
                        ? rtt_gram_normal(op, arm_masks[ai], Q_dev[g], d, Gi, stream)
                        : rtt_gram(op, arm_masks[ai], Q_dev[g], d, Gi, stream);
            }
            if (s == RTT_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
                set_error("rank audit: Gram failed: %s", cudaGetErrorString(cudaGetLastError()));
                s = RTT_ECUDA;
            }
            r.s_ref = op->s_ref;
            const auto t2 = std::chrono::steady_clock::now();
            r.seconds_probe = std::chrono::duration<double>(t1 - t0).count();
            r.seconds_gram = std::chrono::duration<double>(t2 - t1).count();
            r.seconds = std::chrono::duration<double>(t2 - t0).count();
        }
    }
    // all spectra: eigenvalues of every matrix by tridiagonal reduction and
    // bisection (on a copy), then cyclic Jacobi for any matrix with an
    // eigenvalue within the reduction's error bound of the threshold rho^2
    if (s == RTT_OK) {
        const auto t0 = std::chrono::steady_clock::now();
        cudaStream_t st = (cudaStream_t)stream;
        const size_t bytes = (size_t)nb * d * d * 8;
        if (cudaMemcpyAsync(V, G, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            set_error("rank audit: copy failed");
            s = RTT_ECUDA;
        }
        if (s == RTT_OK) s = rtt_eigvals_sym_batched(d, nb, V, ev.data(), stream);
        for (int b = 0; s == RTT_OK && b < nb; ++b) {
            const double rho = ops[b / n_arms]->opt.rho;
            double amax = 0.0;
            for (int i = 0; i < d; ++i) amax = std::fmax(amax, std::fabs(ev[(size_t)b * d + i]));
            const double bound = 64.0 * d * 2.220446049250313e-16 * amax;
            bool near = false;
            for (int i = 0; i < d; ++i) near = near || std::fabs(ev[(size_t)b * d + i] - rho * rho) <= bound;
            sweeps[b] = 0;
            if (near) {  // decide this matrix with the Jacobi spectrum (relative accuracy)
                s = rtt_eig_sym(d, G + (size_t)b * d * d, ev.data() + (size_t)b * d, V, 80,
                                &sweeps[b], stream);
            }
        }
        const double te = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int b = 0; s == RTT_OK && b < nb; ++b) {
            rtt_audit_record& r = out[b];
            std::vector<double> sig(d);
            const double rho = ops[b / n_arms]->opt.rho;
            int rank = 0;
            double margin = INFINITY, smin_pos = INFINITY;
            s = rtt_operational_rank(d, ev.data() + (size_t)b * d, rho, &rank, &margin, sig.data());
            if (s != RTT_OK) break;
            for (int i = 0; i < d; ++i)
                if (sig[i] > 0.0) smin_pos = std::fmin(smin_pos, sig[i]);
            r.rank = rank;
            r.margin = margin;
            r.sigma_max = sig[0];
            r.sigma_min_pos = smin_pos;
            r.jacobi_sweeps = sweeps[b];
            r.seconds += te / nb;
            r.seconds_eig = te / nb;
            if (sigma_out)
                for (int i = 0; i < d; ++i) sigma_out[(size_t)b * d + i] = sig[i];
        }
    }
    cudaFree(G);
    cudaFree(V);
    return s;
}
